// Dense linear algebra of Sec. VI on the device: overlaps (Eq. 5), Cholesky
// orthogonalisation (Eq. 6) and subspace diagonalisation (Eqs. 7-8).
//
// Tall-skinny contractions over grid points:
//   k_gram    S = dV X^T Y, split over blocks of points ("blocks of points",
//             Sec. VI) and accumulated in FP64.  FP64 data: FP64 FMA.  FP32
//             data: every product is formed exactly as a float pair (fma
//             error term) and accumulated as a compensated float pair, so
//             the FP64 result is accurate to ~2^-44 relative while running
//             on the FP32 pipes (FP64 throughput on this part is 1/64 of
//             FP32).
//   k_rowmul  Y = alpha X C + beta Y applied row by row (each CTA owns whole
//             rows), so the in-place update Psi <- Psi C needs no copy.
// Small dense kernels (n <= a few hundred, FP64 unless stated):
//   k_chol    S = U^T U, right-looking, one CTA, status on failure
//   k_trinv   U^-1 by back substitution, one thread per column
//   k_gemm_nn small C = alpha op(A) op(B) + beta C, tiled over many CTAs
//   k_jacobi  cyclic Jacobi with the parallel (round-robin) ordering, one
//             CTA, FP32 or FP64
//   RefSyEv   FP64 refinement of FP32 eigenvectors by the iterative
//             refinement of Ogita & Aishima (2018)
#include <algorithm>
#include <cmath>
#include <vector>

#include "device.h"
#include "linalg.h"

namespace rs {

// ------------------------------------------------------------- k_gram ---

constexpr int G_TM = 64, G_TN = 64, G_TK = 16, G_NT = 256;

// Error-free transformation s + e = a + b (Knuth); the _rn intrinsics keep
// the compiler from contracting any step into a fused multiply-add.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// FP64 data: plain FP64 accumulation.  FP32 data: compensated float pairs.
template <typename T> struct GramAcc;
template <> struct GramAcc<double> {
    double v = 0;
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double value() const { return v; }
};
// FP32 data, plain FP32 accumulation within a chunk of points (the inner
// iterations of the FP32 mode); chunks are combined in FP64.
struct GramAccFast {
    float v = 0;
    __device__ __forceinline__ void add(float a, float b) { v = fmaf(a, b, v); }
    __device__ __forceinline__ double value() const { return (double)v; }
};
template <> struct GramAcc<float> {
    float hi = 0, lo = 0;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -p);   // exact: a*b = p + pe
        float s, e;
        two_sum(hi, p, s, e);
        hi = s;
        lo += e + pe;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// S[i][j] += dV * sum_{p in chunk} X[p][i] Y[p][j]; grid (ceil(nx/64), ceil(ny/64), splits)
template <typename T, typename ACC = GramAcc<T>>
__global__ void __launch_bounds__(G_NT) k_gram(const T *__restrict__ X, int64_t ldx, int nx, const T *__restrict__ Y,
                                               int64_t ldy, int ny, int64_t npts, int64_t chunk, double dV,
                                               double *__restrict__ S, int64_t lds) {
    __shared__ T xs[G_TK][G_TM + 1];
    __shared__ T ys[G_TK][G_TN + 1];
    const int i0 = blockIdx.x * G_TM, j0 = blockIdx.y * G_TN;
    const int64_t p0 = (int64_t)blockIdx.z * chunk;
    const int64_t p1 = min(npts, p0 + chunk);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 4x4 micro tile at (4ty.., 4tx..)
    ACC acc[4][4];
    for (int64_t pk = p0; pk < p1; pk += G_TK) {
        for (int e = threadIdx.x; e < G_TK * G_TM; e += G_NT) {
            const int k = e / G_TM, c = e % G_TM;
            const int64_t p = pk + k;
            xs[k][c] = (p < p1 && i0 + c < nx) ? X[p * ldx + i0 + c] : T(0);
            ys[k][c] = (p < p1 && j0 + c < ny) ? Y[p * ldy + j0 + c] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < G_TK; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = xs[k][4 * ty + u];
                b[u] = ys[k][4 * tx + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v].add(a[u], b[v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + 4 * ty + u, j = j0 + 4 * tx + v;
            if (i < nx && j < ny) atomicAdd(S + (int64_t)i * lds + j, dV * acc[u][v].value());
        }
}

__global__ void k_zero2d(double *S, int64_t lds, int n, int m) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * m; e += (int64_t)gridDim.x * blockDim.x)
        S[(e / m) * lds + e % m] = 0.0;
}

template <typename T>
int gram(const T *X, int64_t ldx, int nx, const T *Y, int64_t ldy, int ny, int64_t npts, double dV, double *S,
         int64_t lds, cudaStream_t st, bool fast) {
    k_zero2d<<<64, 256, 0, st>>>(S, lds, nx, ny);
    RS_LAUNCH_CHECK();
    const int gx = (nx + G_TM - 1) / G_TM, gy = (ny + G_TN - 1) / G_TN;
    // enough CTAs to fill the GPU twice over, each over a contiguous chunk of points
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>((npts + 255) / 256, (152 * 8) / std::max(1, gx * gy)));
    int64_t chunk = (npts + splits - 1) / splits;
    chunk = (chunk + G_TK - 1) / G_TK * G_TK;
    splits = (int)((npts + chunk - 1) / chunk);
    dim3 grid(gx, gy, splits);
    if constexpr (sizeof(T) == 4) {
        if (fast) {
            k_gram<float, GramAccFast><<<grid, G_NT, 0, st>>>(X, ldx, nx, Y, ldy, ny, npts, chunk, dV, S, lds);
            RS_LAUNCH_CHECK();
            return RS_OK;
        }
    }
    k_gram<T><<<grid, G_NT, 0, st>>>(X, ldx, nx, Y, ldy, ny, npts, chunk, dV, S, lds);
    RS_LAUNCH_CHECK();
    return RS_OK;
}
template int gram<double>(const double *, int64_t, int, const double *, int64_t, int, int64_t, double, double *,
                          int64_t, cudaStream_t, bool);
template int gram<float>(const float *, int64_t, int, const float *, int64_t, int, int64_t, double, double *, int64_t,
                         cudaStream_t, bool);

// ----------------------------------------------------------- k_rowmul ---
// Y[p][0:m] = alpha * sum_k X[p][k] C[k][0:m] + beta * Y[p][0:m] for a tile of
// R_ROWS rows per CTA; X rows are staged in shared memory first, so Y may
// alias X (in-place rotation).  C is FP64 [n][ldc] converted on the fly.

constexpr int R_ROWS = 16, R_NT = 256;

template <typename T>
__global__ void __launch_bounds__(R_NT) k_rowmul(const T *X, int64_t ldx, int n, const double *__restrict__ C,
                                                 int64_t ldc, int m, T *Y, int64_t ldy, int64_t npts, T alpha, T beta) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *xs = reinterpret_cast<T *>(smraw);  // [R_ROWS][n]
    const int64_t r0 = (int64_t)blockIdx.x * R_ROWS;
    const int rows = (int)(npts - r0 < R_ROWS ? npts - r0 : R_ROWS);
    for (int e = threadIdx.x; e < R_ROWS * n; e += R_NT) {
        const int r = e / n, k = e % n;
        xs[e] = r < rows ? X[(r0 + r) * ldx + k] : T(0);
    }
    __syncthreads();
    for (int c0 = 0; c0 < m; c0 += R_NT) {
        const int c = c0 + threadIdx.x;
        T acc[R_ROWS];
#pragma unroll
        for (int r = 0; r < R_ROWS; ++r) acc[r] = 0;
        if (c < m) {
            for (int k = 0; k < n; ++k) {
                const T w = (T)__ldg(C + (int64_t)k * ldc + c);
#pragma unroll
                for (int r = 0; r < R_ROWS; ++r) acc[r] += xs[r * n + k] * w;
            }
            for (int r = 0; r < rows; ++r) {
                T *y = Y + (r0 + r) * ldy + c;
                *y = beta == T(0) ? alpha * acc[r] : alpha * acc[r] + beta * *y;
            }
        }
    }
}

template <typename T>
int rowmul(const T *X, int64_t ldx, int n, const double *C, int64_t ldc, int m, T *Y, int64_t ldy, int64_t npts,
           double alpha, double beta, cudaStream_t st) {
    const size_t smem = (size_t)R_ROWS * n * sizeof(T);
    if (smem > 200 * 1024) return fail(RS_EINVAL, "rowmul: n too large");
    if (smem > 48 * 1024) RS_TRY(smem_optin((const void *)k_rowmul<T>, smem));
    const int64_t blocks = (npts + R_ROWS - 1) / R_ROWS;
    k_rowmul<T><<<(unsigned)blocks, R_NT, smem, st>>>(X, ldx, n, C, ldc, m, Y, ldy, npts, (T)alpha, (T)beta);
    RS_LAUNCH_CHECK();
    return RS_OK;
}
template int rowmul<double>(const double *, int64_t, int, const double *, int64_t, int, double *, int64_t, int64_t,
                            double, double, cudaStream_t);
template int rowmul<float>(const float *, int64_t, int, const double *, int64_t, int, float *, int64_t, int64_t, double,
                           double, cudaStream_t);

// ----------------------------------------------------- small dense FP64 ---

// Right-looking Cholesky of the leading n x n block of A (in place): the
// upper triangle receives U with A = U^T U, the strict lower triangle is
// zeroed.  status[0] = 0, or j+1 if pivot j is not finite or not larger
// than rel * (original A_jj).  One CTA; the matrix is worked on in shared
// memory when it fits (IN_SMEM, the path cholesky takes up to
// CHOL_SMEM_MAX), else in global memory (L1/L2 resident).
// Rows are spread over warps and columns over lanes, so no index division.
constexpr int CHOL_MAX = 2048;
constexpr int CHOL_SMEM_MAX = 160;   // n x n FP64 in 200 KB
template <bool IN_SMEM>
__global__ void __launch_bounds__(1024) k_chol(double *Ag, int lda, int n, double rel, int *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double diag0[CHOL_MAX];
    __shared__ double piv;
    __shared__ int bad;
    double *A = IN_SMEM ? reinterpret_cast<double *>(smraw) : Ag;
    const int ld = IN_SMEM ? n : lda;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (IN_SMEM)
        for (int r = warp; r < n; r += nw)
            for (int c = lane; c < n; c += 32) A[r * ld + c] = Ag[(int64_t)r * lda + c];
    __syncthreads();
    for (int j = tid; j < n; j += blockDim.x) diag0[j] = A[(int64_t)j * ld + j];
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d = A[(int64_t)j * ld + j];
            if (!isfinite(d) || !(d > 0.0) || !(d > rel * diag0[j])) {
                bad = j + 1;
                piv = 1.0;
            } else {
                piv = sqrt(d);
            }
            A[(int64_t)j * ld + j] = piv;
        }
        __syncthreads();
        if (bad) break;
        const double inv = 1.0 / piv;
        double *uj = A + (int64_t)j * ld;
        for (int c = j + 1 + tid; c < n; c += blockDim.x) uj[c] *= inv;
        __syncthreads();
        // trailing update A[r][c] -= U[j][r] U[j][c] on the upper triangle, r, c > j
        for (int r = j + 1 + warp; r < n; r += nw) {
            const double ujr = uj[r];
            double *ar = A + (int64_t)r * ld;
            for (int c = r + lane; c < n; c += 32) ar[c] -= ujr * uj[c];
        }
        __syncthreads();
    }
    for (int r = warp; r < n; r += nw)
        for (int c = lane; c < n; c += 32) {
            const double v = c < r ? 0.0 : A[(int64_t)r * ld + c];
            if (IN_SMEM) Ag[(int64_t)r * lda + c] = v;
            else if (c < r) Ag[(int64_t)r * lda + c] = 0.0;
        }
    if (tid == 0) status[0] = bad;
}

// X = U^-1 for upper-triangular U (n x n): one warp per column j, back
// substitution x_i = (delta_ij - sum_{k=i+1..j} U_ik x_k) / U_ii from the
// diagonal upwards, the sums split over the lanes.  X must not alias U.
__global__ void __launch_bounds__(256) k_trinv(const double *__restrict__ U, int ldu, int n, double *__restrict__ X,
                                               int ldx) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int j = blockIdx.x * (blockDim.x >> 5) + wl;
    double *x = reinterpret_cast<double *>(smraw) + (size_t)wl * n;
    if (j >= n) return;
    for (int i = j; i >= 0; --i) {
        const double *ui = U + (int64_t)i * ldu;
        double t = 0.0;
        for (int k = i + 1 + lane; k <= j; k += 32) t += ui[k] * x[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) x[i] = ((i == j ? 1.0 : 0.0) - t) / ui[i];
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) X[(int64_t)i * ldx + j] = i <= j ? x[i] : 0.0;
}

// C = alpha op(A) op(B) + beta C for small dense FP64 matrices (row-major),
// op(X) = X or X^T.  C is m x n, the contraction length is k.  16x16 tiles.
__global__ void k_gemm_small(int m, int n, int k, double alpha, const double *__restrict__ A, int lda, int ta,
                             const double *__restrict__ B, int ldb, int tb, double beta, double *C, int ldc) {
    __shared__ double as[16][17], bs[16][17];
    const int r = blockIdx.y * 16 + threadIdx.y, c = blockIdx.x * 16 + threadIdx.x;
    double acc = 0.0;
    for (int k0 = 0; k0 < k; k0 += 16) {
        const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        const int ar = blockIdx.y * 16 + threadIdx.y, bc = blockIdx.x * 16 + threadIdx.x;
        as[threadIdx.y][threadIdx.x] =
            (ar < m && ka < k) ? (ta ? A[(int64_t)ka * lda + ar] : A[(int64_t)ar * lda + ka]) : 0.0;
        bs[threadIdx.y][threadIdx.x] =
            (kb < k && bc < n) ? (tb ? B[(int64_t)bc * ldb + kb] : B[(int64_t)kb * ldb + bc]) : 0.0;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) acc = fma(as[threadIdx.y][t], bs[t][threadIdx.x], acc);
        __syncthreads();
    }
    if (r < m && c < n) {
        double *y = C + (int64_t)r * ldc + c;
        *y = beta == 0.0 ? alpha * acc : alpha * acc + beta * *y;
    }
}

int gemm_small(int m, int n, int k, double alpha, const double *A, int lda, bool ta, const double *B, int ldb,
               bool tb, double beta, double *C, int ldc, cudaStream_t st) {
    dim3 grid((n + 15) / 16, (m + 15) / 16), blk(16, 16);
    k_gemm_small<<<grid, blk, 0, st>>>(m, n, k, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// Blocked right-looking Cholesky for n > CHOL_SMEM_MAX, block rows of
// CHOL_NB.  The original diagonal, which the pivot test compares against,
// is kept in column 0 of the strict lower triangle (A[j][0], j >= 1: never
// inside a trailing block, and zeroed at the end with the rest of the lower
// triangle).  Per block row k: the diagonal block is factored in shared
// memory (k_chol_diag), the panel U[k][rest] = U_kk^-T A[k][rest] is solved
// by forward substitution, one thread per column (k_chol_panel), and the
// trailing matrix takes A[rest][rest] -= U[k][rest]^T U[k][rest]
// (k_gemm_small; the full square, of which only the upper triangle is read
// later).  status[0] = j+1 of the first failing pivot j; once it is set the
// later diagonal and panel kernels return at once.
constexpr int CHOL_NB = 64;

__global__ void k_chol_save_diag(double *A, int lda, int n) {
    for (int j = 1 + blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        A[(int64_t)j * lda] = A[(int64_t)j * lda + j];
}

// factor the bk x bk diagonal block at (k, k) in shared memory
__global__ void __launch_bounds__(1024) k_chol_diag(double *Ag, int lda, int k, int bk, double rel, int *status) {
    __shared__ double A[CHOL_NB * CHOL_NB];
    __shared__ double piv;
    __shared__ int bad;
    if (*(volatile int *)status) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    double *blk = Ag + (int64_t)k * lda + k;
    for (int r = warp; r < bk; r += nw)
        for (int c = lane; c < bk; c += 32) A[r * bk + c] = blk[(int64_t)r * lda + c];
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < bk; ++j) {
        if (tid == 0) {
            const int g = k + j;
            const double d0 = g == 0 ? A[0] : Ag[(int64_t)g * lda];   // original diagonal (saved)
            const double d = A[j * bk + j];
            if (!isfinite(d) || !(d > 0.0) || !(d > rel * d0)) {
                bad = g + 1;
                piv = 1.0;
            } else {
                piv = sqrt(d);
            }
            A[j * bk + j] = piv;
        }
        __syncthreads();
        if (bad) break;
        const double inv = 1.0 / piv;
        double *uj = A + j * bk;
        for (int c = j + 1 + tid; c < bk; c += blockDim.x) uj[c] *= inv;
        __syncthreads();
        for (int r = j + 1 + warp; r < bk; r += nw) {
            const double ujr = uj[r];
            for (int c = r + lane; c < bk; c += 32) A[r * bk + c] -= ujr * uj[c];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicCAS(status, 0, bad);
        return;
    }
    for (int r = warp; r < bk; r += nw)
        for (int c = r + lane; c < bk; c += 32) blk[(int64_t)r * lda + c] = A[r * bk + c];
}

// panel: rows k..k+bk-1, columns c >= k+bk, x = U_kk^-T a by forward
// substitution, x_i = (a_i - sum_{l<i} U_li x_l) / U_ii, in place
__global__ void __launch_bounds__(128) k_chol_panel(double *Ag, int lda, int n, int k, int bk, const int *status) {
    __shared__ double U[CHOL_NB * CHOL_NB];
    if (*(volatile const int *)status) return;
    const int tid = threadIdx.x;
    const double *blk = Ag + (int64_t)k * lda + k;
    for (int e = tid; e < bk * bk; e += blockDim.x) U[e] = blk[(int64_t)(e / bk) * lda + e % bk];
    __syncthreads();
    const int c = k + bk + blockIdx.x * blockDim.x + tid;
    if (c >= n) return;
    double *col = Ag + (int64_t)k * lda + c;
    double x[CHOL_NB];   // the column's solution, in registers (fully unrolled loops)
#pragma unroll
    for (int i = 0; i < CHOL_NB; ++i) {
        if (i < bk) {
            double t = col[(int64_t)i * lda];
#pragma unroll
            for (int l = 0; l < i; ++l) t -= U[l * bk + i] * x[l];
            t /= U[i * bk + i];
            x[i] = t;
            col[(int64_t)i * lda] = t;
        }
    }
}

__global__ void k_zero_lower(double *A, int lda, int n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e % n);
        if (c < r) A[(int64_t)r * lda + c] = 0.0;
    }
}

int cholesky(double *A, int lda, int n, double rel, int *status_dev, cudaStream_t st) {
    if (n <= CHOL_SMEM_MAX) {
        const size_t sm = sizeof(double) * (size_t)n * n;
        RS_TRY(smem_optin((const void *)k_chol<true>, sm));
        k_chol<true><<<1, 1024, sm, st>>>(A, lda, n, rel, status_dev);
        RS_LAUNCH_CHECK();
        return RS_OK;
    }
    RS_CUDA(cudaMemsetAsync(status_dev, 0, sizeof(int), st));
    k_chol_save_diag<<<(n + 255) / 256, 256, 0, st>>>(A, lda, n);
    RS_LAUNCH_CHECK();
    for (int k = 0; k < n; k += CHOL_NB) {
        const int bk = std::min(CHOL_NB, n - k), m = n - k - bk;
        k_chol_diag<<<1, 1024, 0, st>>>(A, lda, k, bk, rel, status_dev);
        RS_LAUNCH_CHECK();
        if (m == 0) break;
        k_chol_panel<<<(m + 127) / 128, 128, 0, st>>>(A, lda, n, k, bk, status_dev);
        RS_LAUNCH_CHECK();
        double *Xk = A + (int64_t)k * lda + k + bk, *C = A + (int64_t)(k + bk) * lda + k + bk;
        RS_TRY(gemm_small(m, m, bk, -1.0, Xk, lda, true, Xk, lda, false, 1.0, C, lda, st));
    }
    k_zero_lower<<<std::min(1024, (n * n + 255) / 256), 256, 0, st>>>(A, lda, n);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

int tri_inv(const double *U, int ldu, int n, double *X, int ldx, cudaStream_t st) {
    constexpr int WPB = 8;   // columns (warps) per CTA
    const size_t sm = sizeof(double) * (size_t)WPB * n;
    if (sm > 48 * 1024) RS_TRY(smem_optin((const void *)k_trinv, sm));
    k_trinv<<<(n + WPB - 1) / WPB, 32 * WPB, sm, st>>>(U, ldu, n, X, ldx);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// (A + A^T) / 2 in place (n x n)
__global__ void k_symmetrize(double *A, int lda, int n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e % n);
        if (c > r) {
            const double v = 0.5 * (A[(int64_t)r * lda + c] + A[(int64_t)c * lda + r]);
            A[(int64_t)r * lda + c] = v;
            A[(int64_t)c * lda + r] = v;
        }
    }
}

int symmetrize(double *A, int lda, int n, cudaStream_t st) {
    k_symmetrize<<<std::min(1024, (n * n + 255) / 256), 256, 0, st>>>(A, lda, n);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// ----------------------------------------------------------- Jacobi ---
// Cyclic Jacobi eigenvalue iteration for a symmetric n x n matrix (n even).
// Each round applies n/2 rotations on disjoint index pairs (the round-robin
// "circle" ordering: pair (0, 1 + r mod (n-1)) and the pairs
// (1 + (r+k) mod (n-1), 1 + (r-k) mod (n-1)), k = 1..n/2-1), each rotation
// annihilating its (p,q) entry; n-1 rounds make a sweep visiting every pair.
// Matrices whose packed triangle fits one CTA's shared memory use
// k_jacobi_pk below; larger ones the cooperative multi-CTA k_jacobi_grid.

// Multi-CTA variant for matrices too large for one CTA's shared memory
// (cooperative launch: every CTA resident).  A and V stay in global memory
// (L2-resident).  A round has three parts:
//  - Every CTA computes all n/2 rotations of the round.  Their inputs (the
//    diagonal and the pivot entries A[p_k][q_k]) come from a compact buffer
//    that the previous round wrote.
//  - Each warp takes whole units.  An A unit is a pair of rows (p_k, q_k),
//    rotated as rows by (c_k, s_k) and as columns by every (c_l, s_l) in the
//    warp's shared memory (row and column rotations commute in J^T A J).  A
//    V unit is a pair of rows of V, rotated as columns only.  A unit's loads
//    and stores are whole coalesced rows.  The A unit that owns row x also
//    writes the next round's inputs from x: its diagonal entry, and its
//    entry in the next round's pivot if x is that pair's p.  These go to the
//    other half of the double-buffered input, so one grid barrier per round
//    suffices.
//  - A software grid barrier (bounded spin; on timeout err[0] is set and
//    every CTA returns).
// FP32 rotates A - sigma I, sigma the mean of the diagonal (the same
// eigenvectors): its rounding and stopping test then scale with the spread
// of the spectrum, not its offset.
constexpr long long GRID_SPIN_LIMIT = 1ll << 26;

__device__ __forceinline__ bool grid_barrier(unsigned *count, volatile unsigned *gen, unsigned nblocks, int *err) {
    __threadfence();   // every thread publishes its writes before the block arrives
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned my = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            *count = 0;
            __threadfence();
            atomicAdd((unsigned *)gen, 1u);
        } else {
            long long spins = 0;
            while (*gen == my) {
                if (++spins > GRID_SPIN_LIMIT || *(volatile int *)err) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)err == 0;
}


// Single-CTA cyclic Jacobi with the matrix held in shared memory as its
// packed upper triangle (n (n+1)/2 elements), for n up to a few hundred.  A
// round of the circle ordering rotates h = n/2 disjoint pairs (p_k, q_k); the
// two-sided update J^T A J then acts independently on every 2 x 2 block
// A[{p_k,q_k}][{p_l,q_l}] (k <= l), so a round is one pass over those blocks
// between two barriers.  The rotations are logged, (c, s) per pair per round,
// and the eigenvectors are accumulated afterwards by k_jacobi_vacc, whose
// CTAs each own a few rows of V.  On exit w holds the eigenvalues ascending,
// perm[i] the rank of diagonal position i, info[0] the sweeps used (-1 when
// max_sweeps ran out).
__device__ __forceinline__ void circle_pair(int r, int k, int m, int &p, int &q) {
    if (k == 0) {
        p = 0;
        q = 1 + r % m;
    } else {
        p = 1 + (r + k) % m;
        q = 1 + (r - k + m) % m;
    }
}

// Jacobi rotation (c, s) that zeroes a_pq of the 2 x 2 block [[app, apq],
// [apq, aqq]]: t = tan(theta) is the smaller root of t^2 + 2 tau t - 1 = 0,
// tau = (aqq - app) / (2 apq), written t = sign(tau) |2 apq| /
// (|aqq - app| + sqrt((aqq - app)^2 + (2 apq)^2)) (one square root and one
// division on the dependent path), c = 1 / sqrt(1 + t^2) by the reciprocal
// square root with one Newton step, s = t c.  An off-diagonal entry whose
// square underflows is left alone.
template <typename T> __device__ __forceinline__ void jacobi_cs(T app, T aqq, T apq, T &c, T &s) {
    c = T(1);
    s = T(0);
    const T d = aqq - app, a2 = T(2) * apq;
    // an entry whose square underflows is below any rounding of the block:
    // no rotation (and no 0 / 0 when the diagonal entries are equal)
    if (!(a2 * a2 > T(0))) return;
    T t = fabs(a2) / (fabs(d) + sqrt(d * d + a2 * a2));
    if ((d < T(0)) != (a2 < T(0))) t = -t;   // sign(tau) = sign(d) sign(apq)
    const T x = T(1) + t * t;
    T r;
    if constexpr (sizeof(T) == 4) {
        r = rsqrtf(x);
        r = r * (1.5f - 0.5f * x * r * r);
    } else {
        r = T(1) / sqrt(x);
    }
    c = r;
    s = t * r;
}

// shared memory of k_jacobi_grid ahead of its row buffers: (c, s) and
// (p, q) of the n/2 rotations, 16-byte aligned
__host__ __device__ inline size_t jacobi_grid_head_bytes(int n, size_t es) {
    const size_t h = n / 2;
    return (2 * h * es + 2 * h * sizeof(int) + 15) / 16 * 16;
}

// slot of index x in round r of the circle ordering: pair k and whether x
// is that pair's p (x = p_k) or q (x = q_k)
__device__ __forceinline__ void circle_slot(int x, int r, int m, int h, int &k, bool &is_p) {
    if (x == 0) {
        k = 0;
        is_p = true;
        return;
    }
    const int y = x - 1, rr = r % m;
    if (y == rr) {
        k = 0;
        is_p = false;
        return;
    }
    const int d = ((y - rr) % m + m) % m;   // 1 .. m-1
    if (d <= h - 1) {
        k = d;
        is_p = true;
    } else {
        k = m - d;
        is_p = false;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_jacobi_grid(T *A, T *V, int n, int max_sweeps, double tol, double *w,
                                                     double *Vout, int ldv, int *info, unsigned *bar, double *red_g,
                                                     int *err, T *pivots) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int h = n / 2, m = n - 1;
    T *cs = reinterpret_cast<T *>(smraw);
    T *sn = cs + h;
    int *pp = reinterpret_cast<int *>(sn + h);
    int *qq = pp + h;
    const int tid = threadIdx.x, nt = blockDim.x, G = gridDim.x, bid = blockIdx.x;
    const int lane = tid & 31, warp = tid >> 5, W = nt >> 5;
    T *r0 = reinterpret_cast<T *>(smraw + jacobi_grid_head_bytes(n, sizeof(T))) + (size_t)warp * 2 * n;
    T *r1 = r0 + n;
    // round inputs, two halves of (diagonal [n], pivots [h])
    auto diag_of = [&](int half) { return pivots + (size_t)half * (n + h); };
    auto piv_of = [&](int half) { return pivots + (size_t)half * (n + h) + n; };
    __shared__ double red[8];
    unsigned *count = bar;
    volatile unsigned *gen = bar + 1;
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double t = 0;
        if (tid == 0)
            for (int i = 0; i < W; ++i) t += red[i];
        __syncthreads();
        return t;
    };
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = bid * (int64_t)nt + tid; e < nn; e += (int64_t)G * nt) V[e] = (e / n == e % n) ? T(1) : T(0);
    // the shift (FP32): mean of the diagonal, in red_g[max_sweeps + 1]
    double shift = 0;
    if constexpr (sizeof(T) == 4) {
        double d = 0;
        for (int i = bid * nt + tid; i < n; i += G * nt) d += (double)__ldcg(A + (int64_t)i * n + i);
        const double t = block_sum(d);
        if (tid == 0) atomicAdd(red_g + max_sweeps + 1, t);
        if (!grid_barrier(count, gen, G, err)) return;
        shift = *(volatile double *)(red_g + max_sweeps + 1) / n;
    }
    // shifted diagonal, round 0's inputs, and the Frobenius norm of the
    // unshifted matrix (red_g[0]), against which the stopping test measures
    // the off-diagonal part: inside the FP32 eigensolver's subspace steps a
    // tighter test (the shifted norm) keeps rotating by couplings that an FP32
    // Jacobi resolves only to about 1e-3 of a column, and those rotations
    // stalled the 300-atom solve at that residual
    double loc = 0;
    for (int64_t e = bid * (int64_t)nt + tid; e < nn; e += (int64_t)G * nt) {
        T x = __ldcg(A + e);
        loc += (double)x * (double)x;
        const int i = (int)(e / n);
        if (i == (int)(e % n)) {
            x = (T)((double)x - shift);
            A[e] = x;
            diag_of(0)[i] = x;
        }
    }
    for (int k = bid * nt + tid; k < h; k += G * nt) {
        int p, q;
        circle_pair(0, k, m, p, q);
        piv_of(0)[k] = __ldcg(A + (int64_t)p * n + q);
    }
    {
        const double f = block_sum(loc);
        if (tid == 0) atomicAdd(red_g, f);
    }
    if (!grid_barrier(count, gen, G, err)) return;
    const double fro2 = *(volatile double *)red_g;
    int sweep = 0, done = 0;
    int64_t t = 0;   // rounds taken: round t reads half t % 2 of the inputs and writes the other
    for (; sweep < max_sweeps; ++sweep) {
        loc = 0;
        for (int64_t e = bid * (int64_t)nt + tid; e < nn; e += (int64_t)G * nt)
            if (e / n != e % n) loc += (double)__ldcg(A + e) * (double)__ldcg(A + e);
        const double o = block_sum(loc);
        if (tid == 0) atomicAdd(red_g + 1 + sweep, o);
        if (!grid_barrier(count, gen, G, err)) return;
        if (*(volatile double *)(red_g + 1 + sweep) <= tol * tol * fro2) {
            done = 1;
            break;
        }
        for (int r = 0; r < m; ++r, ++t) {
            const int cur = (int)(t & 1), nxt = cur ^ 1;
            const T *dg = diag_of(cur), *pv = piv_of(cur);
            for (int k = tid; k < h; k += nt) {
                int p, q;
                circle_pair(r, k, m, p, q);
                T c, s_;
                if constexpr (sizeof(T) == 4) {
                    // t = tan(theta) in FP32 (it only has to annihilate the
                    // pivot to FP32 accuracy); c = (1 + t^2)^-1/2 and s = t c
                    // from an FP64 reciprocal square root, rounded once: in
                    // FP32 the reciprocal square root and its Newton step leave
                    // c^2 + s^2 off 1 by a biased fraction of an ulp, which the
                    // n rotations of a round compound.  Every CTA computes all
                    // n/2 rotations, so their FP64 work is kept to one rsqrt.
                    const float app = __ldcg(dg + p), aqq = __ldcg(dg + q), apq = __ldcg(pv + k);
                    const float d = aqq - app, a2 = 2.f * apq;
                    c = 1.f;
                    s_ = 0.f;
                    if (a2 * a2 > 0.f) {
                        float tt = fabsf(a2) / (fabsf(d) + sqrtf(d * d + a2 * a2));
                        if ((d < 0.f) != (a2 < 0.f)) tt = -tt;
                        const double r = rsqrt(1.0 + (double)tt * (double)tt);
                        c = (float)r;
                        s_ = (float)((double)tt * r);
                    }
                } else {
                    jacobi_cs<T>(__ldcg(dg + p), __ldcg(dg + q), __ldcg(pv + k), c, s_);
                }
                cs[k] = c;
                sn[k] = s_;
                pp[k] = p;
                qq[k] = q;
            }
            __syncthreads();
            const int rn = (r + 1) % m;   // the next round (round 0 of the next sweep after the last)
            for (int u = bid * W + warp; u < 2 * h; u += G * W) {
                const bool is_a = u < h;
                const int p = is_a ? pp[u] : 2 * (u - h), q = is_a ? qq[u] : 2 * (u - h) + 1;
                T *x0 = (is_a ? A : V) + (int64_t)p * n, *x1 = (is_a ? A : V) + (int64_t)q * n;
                if (is_a) {
                    const T c = cs[u], s_ = sn[u];
                    for (int j = lane; j < n; j += 32) {
                        const T a = __ldcg(x0 + j), b = __ldcg(x1 + j);
                        r0[j] = c * a - s_ * b;
                        r1[j] = s_ * a + c * b;
                    }
                } else {
                    for (int j = lane; j < n; j += 32) {
                        r0[j] = __ldcg(x0 + j);
                        r1[j] = __ldcg(x1 + j);
                    }
                }
                __syncwarp();
                for (int l = lane; l < h; l += 32) {
                    const int P = pp[l], Q = qq[l];
                    const T c = cs[l], s_ = sn[l];
                    T a = r0[P], b = r0[Q];
                    r0[P] = c * a - s_ * b;
                    r0[Q] = s_ * a + c * b;
                    a = r1[P];
                    b = r1[Q];
                    r1[P] = c * a - s_ * b;
                    r1[Q] = s_ * a + c * b;
                }
                __syncwarp();
                if (is_a && lane == 0) {
                    r0[q] = T(0);   // the annihilated pivot
                    r1[p] = T(0);
                    for (int side = 0; side < 2; ++side) {
                        const int x = side ? q : p;
                        const T *rx = side ? r1 : r0;
                        diag_of(nxt)[x] = rx[x];
                        int k2, p2, q2;
                        bool is_p;
                        circle_slot(x, rn, m, h, k2, is_p);
                        if (is_p) {
                            circle_pair(rn, k2, m, p2, q2);
                            piv_of(nxt)[k2] = rx[q2];
                        }
                    }
                }
                __syncwarp();
                for (int j = lane; j < n; j += 32) {
                    x0[j] = r0[j];
                    x1[j] = r1[j];
                }
                __syncwarp();
            }
            if (!grid_barrier(count, gen, G, err)) return;
        }
    }
    // ascending order (ties by index), outputs split over CTAs
    for (int i = bid * nt + tid; i < n; i += G * nt) {
        const T di = __ldcg(A + (int64_t)i * n + i);
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const T dj = __ldcg(A + (int64_t)j * n + j);
            rk += (dj < di) || (dj == di && j < i);
        }
        w[rk] = (double)di + shift;
        for (int k = 0; k < n; ++k) Vout[(int64_t)k * ldv + rk] = (double)__ldcg(V + (int64_t)k * n + i);
    }
    if (bid == 0 && tid == 0) info[0] = done ? sweep : -1;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_jacobi_pk(const double *__restrict__ Ag, int lda, int n, int max_sweeps,
                                                    double tol, T *__restrict__ rot, double *__restrict__ w,
                                                    int *__restrict__ perm, int *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int h = n / 2, m = n - 1;
    T *cs = reinterpret_cast<T *>(smraw);
    T *sn = cs + h;
    T *a = sn + h;
    const int npk = n * (n + 1) / 2;
    int *ro = reinterpret_cast<int *>(a + npk);   // packed offset of row i minus i: f(i,j) = ro[i] + j, i <= j
    int *pp = ro + n;
    int *qq = pp + h;
    __shared__ double red[32];
    __shared__ double fro2, off2;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    __shared__ double shift;
    for (int i = tid; i < n; i += nt) ro[i] = i * (2 * n - i - 1) / 2;
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double t = 0;
        if (tid < 32) {
            t = tid < nw ? red[tid] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        }
        return t;  // valid in thread 0
    };
    // FP32: rotate A - sigma I, sigma the mean of the diagonal (the same
    // eigenvectors), so that the rounding of the rotations and the stopping
    // test scale with the spread of the spectrum rather than its offset
    {
        double d = 0;
        if constexpr (sizeof(T) == 4)
            for (int i = tid; i < n; i += nt) d += Ag[(int64_t)i * lda + i];
        const double t = block_sum(d);
        if (tid == 0) shift = t / n;
    }
    __syncthreads();
    for (int i = warp; i < n; i += nw)
        for (int j = i + lane; j < n; j += 32)
            a[ro[i] + j] = (T)(j == i ? Ag[(int64_t)i * lda + j] - shift : Ag[(int64_t)i * lda + j]);
    __syncthreads();
    {
        double d = 0, o = 0;
        for (int i = warp; i < n; i += nw)
            for (int j = i + lane; j < n; j += 32) {
                const double x = (double)a[ro[i] + j];
                if (j == i) d += x * x;
                else o += x * x;
            }
        const double f = block_sum(d + 2.0 * o);
        if (tid == 0) fro2 = f;
    }
    __syncthreads();
    int sweep = 0, done = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double o = 0;
        for (int i = warp; i < n; i += nw)
            for (int j = i + 1 + lane; j < n; j += 32) {
                const double x = (double)a[ro[i] + j];
                o += x * x;
            }
        const double t = block_sum(2.0 * o);
        if (tid == 0) off2 = t;
        __syncthreads();
        if (off2 <= tol * tol * fro2) {
            done = 1;
            break;
        }
        for (int r = 0; r < m; ++r) {
            for (int k = tid; k < h; k += nt) {
                int p, q;
                circle_pair(r, k, m, p, q);
                const int lo = min(p, q), hi = max(p, q);
                T c, s_;
                jacobi_cs(a[ro[p] + p], a[ro[q] + q], a[ro[lo] + hi], c, s_);
                cs[k] = c;
                sn[k] = s_;
                pp[k] = p;
                qq[k] = q;
                T *lg = rot + 2 * (((int64_t)sweep * m + r) * h + k);
                lg[0] = c;
                lg[1] = s_;
            }
            __syncthreads();
            for (int k = warp; k < h; k += nw) {
                const int pk = pp[k], qk = qq[k];
                const T ck = cs[k], sk = sn[k];
                for (int l = k + lane; l < h; l += 32) {
                    const int pl = pp[l], ql = qq[l];
                    const T cl = cs[l], sl = sn[l];
                    if (l == k) {
                        const int lo = min(pk, qk), hi = max(pk, qk);
                        const T app = a[ro[pk] + pk], aqq = a[ro[qk] + qk], apq = a[ro[lo] + hi];
                        // rows then columns of [[app, apq], [apq, aqq]]
                        const T x00 = ck * app - sk * apq, x01 = ck * apq - sk * aqq;
                        const T x10 = sk * app + ck * apq, x11 = sk * apq + ck * aqq;
                        a[ro[pk] + pk] = ck * x00 - sk * x01;
                        a[ro[qk] + qk] = sk * x10 + ck * x11;
                        a[ro[lo] + hi] = T(0);
                    } else {
                        auto at = [&](int i, int j) -> T & { return i <= j ? a[ro[i] + j] : a[ro[j] + i]; };
                        T &b00 = at(pk, pl), &b01 = at(pk, ql), &b10 = at(qk, pl), &b11 = at(qk, ql);
                        const T x00 = ck * b00 - sk * b10, x10 = sk * b00 + ck * b10;
                        const T x01 = ck * b01 - sk * b11, x11 = sk * b01 + ck * b11;
                        b00 = cl * x00 - sl * x01;
                        b01 = sl * x00 + cl * x01;
                        b10 = cl * x10 - sl * x11;
                        b11 = sl * x10 + cl * x11;
                    }
                }
            }
            __syncthreads();
        }
    }
    // ascending order (ties by index)
    for (int i = tid; i < n; i += nt) {
        const T di = a[ro[i] + i];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const T dj = a[ro[j] + j];
            rk += (dj < di) || (dj == di && j < i);
        }
        perm[i] = rk;
        w[rk] = (double)di + shift;
    }
    if (tid == 0) info[0] = done ? sweep : -1;
}

// Single-CTA cyclic Jacobi for FP32 with the full matrix in shared memory
// (row stride n + 1, so that a warp's accesses along a row and down a column
// fall in distinct banks), for orders whose full matrix fits.  Same circle
// ordering, rotation log, eigenvalue order and outputs as k_jacobi_pk; a
// round applies the h disjoint rotations as J^T A (rows p, q of every pair,
// all columns) and then A J (columns p, q, all rows), one warp per pair.
template <typename T>
__global__ void __launch_bounds__(1024) k_jacobi_full(const double *__restrict__ Ag, int lda, int n, int max_sweeps,
                                                      double tol, T *__restrict__ rot, double *__restrict__ w,
                                                      int *__restrict__ perm, int *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int h = n / 2, m = n - 1, ld = n + 1;
    T *cs = reinterpret_cast<T *>(smraw);
    T *sn = cs + h;
    int *pp = reinterpret_cast<int *>(sn + h);
    int *qq = pp + h;
    T *a = reinterpret_cast<T *>(qq + h);
    __shared__ double red[32];
    __shared__ double fro2, off2, shift;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double t = 0;
        if (tid < 32) {
            t = tid < nw ? red[tid] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        }
        return t;  // valid in thread 0
    };
    // rotate A - sigma I, sigma the mean of the diagonal (see k_jacobi_pk)
    {
        double d = 0;
        for (int i = tid; i < n; i += nt) d += Ag[(int64_t)i * lda + i];
        const double t = block_sum(d);
        if (tid == 0) shift = t / n;
    }
    __syncthreads();
    for (int i = warp; i < n; i += nw)
        for (int j = lane; j < n; j += 32)
            a[i * ld + j] = (T)(j == i ? Ag[(int64_t)i * lda + j] - shift : Ag[(int64_t)i * lda + j]);
    __syncthreads();
    {
        double f = 0;
        for (int i = warp; i < n; i += nw)
            for (int j = lane; j < n; j += 32) {
                const double x = (double)a[i * ld + j];
                f += x * x;
            }
        const double t = block_sum(f);
        if (tid == 0) fro2 = t;
    }
    __syncthreads();
    int sweep = 0, done = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double o = 0;
        for (int i = warp; i < n; i += nw)
            for (int j = lane; j < n; j += 32)
                if (j != i) {
                    const double x = (double)a[i * ld + j];
                    o += x * x;
                }
        const double t = block_sum(o);
        if (tid == 0) off2 = t;
        __syncthreads();
        if (off2 <= tol * tol * fro2) {
            done = 1;
            break;
        }
        for (int r = 0; r < m; ++r) {
            for (int k = tid; k < h; k += nt) {
                int p, q;
                circle_pair(r, k, m, p, q);
                T c, s_;
                jacobi_cs(a[p * ld + p], a[q * ld + q], a[p * ld + q], c, s_);
                cs[k] = c;
                sn[k] = s_;
                pp[k] = p;
                qq[k] = q;
                T *lg = rot + 2 * (((int64_t)sweep * m + r) * h + k);
                lg[0] = c;
                lg[1] = s_;
            }
            __syncthreads();
            // rows p, q of every pair
            for (int k = warp; k < h; k += nw) {
                const int p = pp[k], q = qq[k];
                const T c = cs[k], s_ = sn[k];
                T *rp = a + p * ld, *rq = a + q * ld;
                for (int j = lane; j < n; j += 32) {
                    const T x = rp[j], y = rq[j];
                    rp[j] = c * x - s_ * y;
                    rq[j] = s_ * x + c * y;
                }
            }
            __syncthreads();
            // columns p, q of every pair; the pair's own off-diagonal entry is zero
            for (int k = warp; k < h; k += nw) {
                const int p = pp[k], q = qq[k];
                const T c = cs[k], s_ = sn[k];
                for (int j = lane; j < n; j += 32) {
                    T *rj = a + j * ld;
                    const T x = rj[p], y = rj[q];
                    rj[p] = (j == q) ? T(0) : c * x - s_ * y;
                    rj[q] = (j == p) ? T(0) : s_ * x + c * y;
                }
            }
            __syncthreads();
        }
    }
    // ascending order (ties by index)
    for (int i = tid; i < n; i += nt) {
        const T di = a[i * ld + i];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const T dj = a[j * ld + j];
            rk += (dj < di) || (dj == di && j < i);
        }
        perm[i] = rk;
        w[rk] = (double)di + shift;
    }
    if (tid == 0) info[0] = done ? sweep : -1;
}

// V = product of the logged rotations, row by row: CTA b owns rows
// [RB b, RB b + RB) in shared memory (identity at the start); thread k applies
// pair k's rotation of every round.  Vout[i][perm[j]] = V[i][j] (FP64).
constexpr int VACC_RB = 8;
template <typename T>
__global__ void k_jacobi_vacc(const T *__restrict__ rot, int n, int max_sweeps, const int *__restrict__ info,
                              const int *__restrict__ perm, double *__restrict__ Vout, int ldv) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *v = reinterpret_cast<T *>(smraw);   // [VACC_RB][n]
    const int h = n / 2, m = n - 1, tid = threadIdx.x;
    const int i0 = blockIdx.x * VACC_RB, nr = min(VACC_RB, n - i0);
    for (int e = tid; e < VACC_RB * n; e += blockDim.x) {
        const int r = e / n, j = e - r * n;
        v[e] = (i0 + r == j) ? T(1) : T(0);
    }
    __syncthreads();
    const int sweeps = info[0] < 0 ? max_sweeps : info[0];
    const int64_t rounds = (int64_t)sweeps * m;
    // the rotations of rounds R .. R + 3 are in flight (log reads hidden
    // behind three rounds of work)
    constexpr int PF = 4;
    T cq[PF], sq[PF];
#pragma unroll
    for (int i = 0; i < PF; ++i) {
        cq[i] = 1;
        sq[i] = 0;
        if (tid < h && i < rounds) {
            cq[i] = rot[2 * (i * h + tid)];
            sq[i] = rot[2 * (i * h + tid) + 1];
        }
    }
    for (int64_t R0 = 0; R0 < rounds; R0 += PF) {
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int64_t R = R0 + i;
            if (R >= rounds) break;
            const T c = cq[i], s_ = sq[i];
            if (tid < h && R + PF < rounds) {
                const T *lg = rot + 2 * ((R + PF) * h + tid);
                cq[i] = lg[0];
                sq[i] = lg[1];
            }
            if (tid < h) {
                int p, q;
                circle_pair((int)(R % m), tid, m, p, q);
#pragma unroll
                for (int r = 0; r < VACC_RB; ++r) {
                    T *row = v + r * n;
                    const T va = row[p], vb = row[q];
                    row[p] = c * va - s_ * vb;
                    row[q] = s_ * va + c * vb;
                }
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < nr * n; e += blockDim.x) {
        const int r = e / n, j = e - r * n;
        Vout[(int64_t)(i0 + r) * ldv + perm[j]] = (double)v[r * n + j];
    }
}

// shared memory of k_jacobi_pk for order n and element type size es
size_t jacobi_pk_smem(int n, size_t es) {
    const size_t h = n / 2;
    return es * (2 * h + (size_t)n * (n + 1) / 2) + sizeof(int) * ((size_t)n + 2 * h) + 64;
}
constexpr size_t JACOBI_PK_MAX_SMEM = 220 * 1024;
// shared memory of k_jacobi_full (row stride n + 1)
size_t jacobi_full_smem(int n, size_t es) {
    const size_t h = n / 2;
    return es * (2 * h + (size_t)n * (n + 1)) + sizeof(int) * 2 * h + 64;
}
// (c, s) entries of the rotation log of up to max_sweeps sweeps
size_t jacobi_log_elems(int n, int max_sweeps) { return 2 * (size_t)max_sweeps * (n - 1) * (n / 2); }

// scratch bytes of jacobi<T> (es = sizeof(T)) for order n and max_sweeps
size_t jacobi_scratch_bytes(int n, int max_sweeps, size_t es) {
    if (jacobi_pk_smem(n, es) <= JACOBI_PK_MAX_SMEM)
        return es * jacobi_log_elems(n, max_sweeps) + sizeof(int) * (size_t)n + 64;
    return 2 * es * (size_t)n * n + 16 + sizeof(double) * ((size_t)max_sweeps + 2) + 16 + 2 * es * ((size_t)n + n / 2) +
           64;
}

// FP64 -> T copy of an n x n matrix into a dense buffer
template <typename T> __global__ void k_copy_cast(const double *A, int lda, int n, T *B) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x)
        B[e] = (T)A[(e / n) * lda + e % n];
}

template <typename T>
int jacobi(const double *A, int lda, int n, int max_sweeps, double tol, double *w, double *V, int ldv, int *info,
           void *scratch, cudaStream_t st) {
    if (n % 2) return fail(RS_EINVAL, "jacobi: n must be even");
    const size_t pk = jacobi_pk_smem(n, sizeof(T));
    if (pk <= JACOBI_PK_MAX_SMEM) {
        // rotation log and rank array in the scratch
        T *rot = reinterpret_cast<T *>(scratch);
        int *perm = reinterpret_cast<int *>(rot + jacobi_log_elems(n, max_sweeps));
        const size_t fs = jacobi_full_smem(n, sizeof(T));
        if (sizeof(T) == 4 && fs <= JACOBI_PK_MAX_SMEM) {
            RS_TRY(smem_optin((const void *)k_jacobi_full<T>, fs));
            k_jacobi_full<T><<<1, 1024, fs, st>>>(A, lda, n, max_sweeps, tol, rot, w, perm, info);
        } else {
            RS_TRY(smem_optin((const void *)k_jacobi_pk<T>, pk));
            k_jacobi_pk<T><<<1, 1024, pk, st>>>(A, lda, n, max_sweeps, tol, rot, w, perm, info);
        }
        RS_LAUNCH_CHECK();
        const int threads = std::max(32, ((n / 2 + 31) / 32) * 32);
        const size_t vs = (size_t)VACC_RB * n * sizeof(T);
        k_jacobi_vacc<T><<<(n + VACC_RB - 1) / VACC_RB, threads, vs, st>>>(rot, n, max_sweeps, info, perm, V, ldv);
        RS_LAUNCH_CHECK();
        return RS_OK;
    }
    T *a = reinterpret_cast<T *>(scratch);
    T *v = a + (size_t)n * n;
    k_copy_cast<T><<<std::min(1024, (n * n + 255) / 256), 256, 0, st>>>(A, lda, n, a);
    RS_LAUNCH_CHECK();
    // grid variant: barrier words, reduction slots, the error flag and the
    // double-buffered round inputs follow V in the scratch
    unsigned *bar = reinterpret_cast<unsigned *>(v + (size_t)n * n);
    double *red_g = reinterpret_cast<double *>(bar + 4);
    int *err = reinterpret_cast<int *>(red_g + max_sweeps + 2);
    T *pivots = reinterpret_cast<T *>(reinterpret_cast<char *>(err) + 16);
    RS_CUDA(cudaMemsetAsync(bar, 0, 16 + sizeof(double) * (max_sweeps + 2) + 16, st));
    // row buffers: two rows of n per warp, at most 8 warps, within 200 KB
    const size_t head = jacobi_grid_head_bytes(n, sizeof(T)), per_warp = 2 * (size_t)n * sizeof(T);
    const int W = (int)std::min<size_t>(8, (200 * 1024 - head) / per_warp);
    if (W < 1) return fail(RS_EINVAL, "jacobi: order %d too large for the multi-CTA variant", n);
    const size_t smem = head + (size_t)W * per_warp;
    RS_TRY(smem_optin((const void *)k_jacobi_grid<T>, smem));
    int nsm = 0, dev = 0, per_sm = 0;
    RS_CUDA(cudaGetDevice(&dev));
    RS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_grid<T>, 32 * W, smem));
    if (per_sm < 1) return fail(RS_ECUDA, "jacobi: the multi-CTA variant cannot be resident");
    // one unit (a row pair of A or of V) per warp and round
    const int G = std::max(1, std::min(nsm * per_sm, (n + W - 1) / W));
    void *args[] = {&a, &v, &n, &max_sweeps, &tol, &w, &V, &ldv, &info, &bar, &red_g, &err, &pivots};
    RS_CUDA(cudaLaunchCooperativeKernel((const void *)k_jacobi_grid<T>, dim3(G), dim3(32 * W), args, smem, st));
    RS_LAUNCH_CHECK();
    return RS_OK;
}
template int jacobi<float>(const double *, int, int, int, double, double *, double *, int, int *, void *, cudaStream_t);
template int jacobi<double>(const double *, int, int, int, double, double *, double *, int, int *, void *,
                            cudaStream_t);

// ---------------------------------------------------------- RefSyEv ---
// One refinement step of approximate eigenvectors X (n x n, FP64) of the
// symmetric A (Ogita & Aishima 2018): with R = I - X^T X and S = X^T A X,
// lambda_i = s_ii / (1 - r_ii) and the correction X <- X (I + E),
//   E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)  if |lambda_i - lambda_j| > delta
//   E_ij = r_ij / 2                                        otherwise,
// delta = 2 (||S - diag(lambda)|| + ||A|| ||R||) (Frobenius norms bound the 2-norms).
__global__ void k_refsyev_norms(const double *A, int lda, const double *R, const double *S, int n, double *out) {
    __shared__ double red[3][32];
    double a = 0, r = 0, s = 0;
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const double av = A[(int64_t)i * lda + j];
        a += av * av;
        r += R[e] * R[e];
        if (i != j) s += S[e] * S[e];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        r += __shfl_down_sync(0xffffffffu, r, o);
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = r;
        red[2][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w)
            for (int q = 0; q < 3; ++q) t[q] += red[q][w];
        // S - diag(lambda): off-diagonal part plus the tiny diagonal residue (ignored)
        out[0] = 2.0 * (sqrt(t[2]) + sqrt(t[0]) * sqrt(t[1]));
    }
}

__global__ void k_refsyev_e(const double *R, const double *S, int n, const double *delta, double *E, double *lam) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const double li = S[(int64_t)i * n + i] / (1.0 - R[(int64_t)i * n + i]);
        const double lj = S[(int64_t)j * n + j] / (1.0 - R[(int64_t)j * n + j]);
        double v;
        if (i == j) {
            v = 0.5 * R[e];
            lam[i] = li;
        } else if (fabs(li - lj) > delta[0]) {
            v = (S[e] + lj * R[e]) / (lj - li);
        } else {
            v = 0.5 * R[e];
        }
        E[e] = v;
    }
}

__global__ void k_add_inplace(double *X, int ldx, const double *D, int ldd, int n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x)
        X[(e / n) * ldx + e % n] += D[(e / n) * ldd + e % n];
}

__global__ void k_identity_minus(double *R, int n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x)
        R[e] = ((e / n == e % n) ? 1.0 : 0.0) - R[e];
}

// X (n x ldx) refined in place; lam[n] receives the refined eigenvalues.
// work: 4 n^2 + 1 doubles.
int refsyev(const double *A, int lda, double *X, int ldx, int n, double *lam, double *work, int iters, cudaStream_t st) {
    double *R = work, *AX = R + (size_t)n * n, *S = AX + (size_t)n * n, *E = S + (size_t)n * n,
           *delta = E + (size_t)n * n;
    const int eb = std::min(1024, (n * n + 255) / 256);
    for (int it = 0; it < iters; ++it) {
        RS_TRY(gemm_small(n, n, n, 1.0, X, ldx, true, X, ldx, false, 0.0, R, n, st));
        k_identity_minus<<<eb, 256, 0, st>>>(R, n);
        RS_TRY(gemm_small(n, n, n, 1.0, A, lda, false, X, ldx, false, 0.0, AX, n, st));
        RS_TRY(gemm_small(n, n, n, 1.0, X, ldx, true, AX, n, false, 0.0, S, n, st));
        k_refsyev_norms<<<1, 1024, 0, st>>>(A, lda, R, S, n, delta);
        k_refsyev_e<<<eb, 256, 0, st>>>(R, S, n, delta, E, lam);
        // X <- X + X E  (via AX as the product buffer)
        RS_TRY(gemm_small(n, n, n, 1.0, X, ldx, false, E, n, false, 0.0, AX, n, st));
        k_add_inplace<<<eb, 256, 0, st>>>(X, ldx, AX, n, n);
        RS_LAUNCH_CHECK();
    }
    return RS_OK;
}

// ------------------------------------------------------------- eigh ---

__global__ void k_pad_copy(const double *A, int lda, int n, int ne, double *B, double big) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ne * ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ne), j = (int)(e % ne);
        B[e] = (i < n && j < n) ? A[(int64_t)i * lda + j] : (i == j ? big : 0.0);
    }
}

__global__ void k_pad_big(const double *A, int lda, int n, double *big) {
    __shared__ double red[32];
    double m = 0;
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        const double v = A[(e / n) * lda + e % n];
        m += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        big[0] = 2.0 * sqrt(t) + 1.0;   // above every eigenvalue of A
    }
}

__global__ void k_copy_block(const double *A, int lda, int m, int n, double *B, int ldb) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
         e += (int64_t)gridDim.x * blockDim.x)
        B[(e / n) * ldb + e % n] = A[(e / n) * lda + e % n];
}

// Jacobi scratch of eigh: FP32 (30 sweeps) or FP64 (60 sweeps) on the padded
// order, the FP64 polish (10 sweeps) on n
static size_t eigh_jacobi_bytes(int n) {
    const int ne = n + (n & 1);
    return std::max({jacobi_scratch_bytes(ne, 30, sizeof(float)), jacobi_scratch_bytes(ne, 60, sizeof(double)),
                     jacobi_scratch_bytes(n + (n & 1), 10, sizeof(double))});
}

size_t eigh_work_bytes(int n) {
    const size_t ne = (size_t)n + (n & 1);
    // padded A, Jacobi vectors, eigenvalues, refinement (4 n^2 + 1), scalars, Jacobi scratch
    return sizeof(double) * (ne * ne * 2 + ne + 4 * (size_t)n * n + 192) + eigh_jacobi_bytes(n);
}

int eigh(const double *A, int lda, int n, double *w, double *V, int ldv, int refine, int *info_dev, void *work,
         cudaStream_t st) {
    const int ne = n + (n & 1);
    double *Ap = reinterpret_cast<double *>(work);
    double *Vp = Ap + (size_t)ne * ne;
    double *wp = Vp + (size_t)ne * ne;
    double *rwork = wp + ne;
    double *big = rwork + 4 * (size_t)n * n + 1;
    double *jscr = big + 64;
    const int eb = std::min(1024, (ne * ne + 255) / 256);
    if (ne != n) {
        k_pad_big<<<1, 1024, 0, st>>>(A, lda, n, big);
        RS_LAUNCH_CHECK();
    }
    // the pad entry's value is read on the device through `big`
    k_pad_copy<<<eb, 256, 0, st>>>(A, lda, n, ne, Ap, 0.0);
    RS_LAUNCH_CHECK();
    if (ne != n) {
        k_copy_block<<<1, 32, 0, st>>>(big, 1, 1, 1, Ap + (size_t)(ne - 1) * ne + (ne - 1), 1);
        RS_LAUNCH_CHECK();
    }
    // FP32 stops at its rounding floor (~u sqrt(n) of the Frobenius norm); FP64
    // at 1e-13 of it
    const double tol32 = std::max(2e-6, 2.4e-7 * std::sqrt((double)ne));
    if (refine != 0) {
        RS_TRY(jacobi<float>(Ap, ne, ne, 30, tol32, wp, Vp, ne, info_dev, jscr, st));
    } else {
        RS_TRY(jacobi<double>(Ap, ne, ne, 60, 1e-13, wp, Vp, ne, info_dev, jscr, st));
    }
    // leading n x n block: eigenvectors of A (the pad entry is decoupled and sorts last)
    k_copy_block<<<eb, 256, 0, st>>>(Vp, ne, n, n, V, ldv);
    k_copy_block<<<1, 256, 0, st>>>(wp, ne, 1, n, w, n);
    RS_LAUNCH_CHECK();
    if (refine <= 0) return RS_OK;
    RS_TRY(refsyev(A, lda, V, ldv, n, w, rwork, refine, st));
    if (n & 1) return RS_OK;
    const size_t nn = (size_t)n * n;
    double *AX = rwork, *B = rwork + nn, *Q = rwork + 2 * nn, *T = rwork + 3 * nn;
    // make V orthonormal to FP64 accuracy (V^T V = U^T U, V <- V U^-1), so that
    // B = V^T A V has exactly the eigenvalues of A ...
    RS_TRY(gemm_small(n, n, n, 1.0, V, ldv, true, V, ldv, false, 0.0, B, n, st));
    RS_TRY(symmetrize(B, n, n, st));
    RS_TRY(cholesky(B, n, n, 0.0, info_dev, st));
    RS_TRY(tri_inv(B, n, n, Q, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, V, ldv, false, Q, n, false, 0.0, T, n, st));
    k_copy_block<<<eb, 256, 0, st>>>(T, n, n, n, V, ldv);
    RS_LAUNCH_CHECK();
    // ... and diagonalise B, which is diagonal up to the couplings the FP32
    // start and the refinement left, with FP64 Jacobi: V <- V Q, B = Q diag(w) Q^T
    RS_TRY(gemm_small(n, n, n, 1.0, A, lda, false, V, ldv, false, 0.0, AX, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, V, ldv, true, AX, n, false, 0.0, B, n, st));
    RS_TRY(symmetrize(B, n, n, st));
    RS_TRY(jacobi<double>(B, n, n, 10, 1e-13, w, Q, n, info_dev, jscr, st));
    RS_TRY(gemm_small(n, n, n, 1.0, V, ldv, false, Q, n, false, 0.0, T, n, st));
    k_copy_block<<<eb, 256, 0, st>>>(T, n, n, n, V, ldv);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

}  // namespace rs

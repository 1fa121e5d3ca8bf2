// Block conjugate-gradient eigensolver (rs_solver_*, rs_eigensolver_step).
//
// The paper's eigensolver is RMM-DIIS working on blocks of orbitals with a
// filter preconditioner (Sec. III) and per-block convergence (Sec. VIII).
// This solver is LOBPCG (Knyazev 2001) applied block by block, followed by
// the orthogonalisation and subspace diagonalisation of Sec. VI after every
// sweep.  For each block X of nb states:
//   lambda = <x|Hx>/<x|x>, R = HX - X lambda, ||r|| (FP64);  a block whose
//   states all satisfy ||r|| <= tol is left alone (Sec. VIII);
//   W = K R (preconditioner);  Y = [W, P] orthogonalised against the states
//   up to and including the block by classical Gram-Schmidt done twice, its
//   columns normalised;  Rayleigh-Ritz on Z = [X, Y] with FP64 Gram matrices
//   (Cholesky with P dropped when the Gram matrix is ill-conditioned);
//   X <- Z C, P <- Z[:, nb:] C[nb:, :].
// After the sweep P follows Psi through U^-1 and xi.
// Precision: RS_F64 keeps everything in FP64.  RS_F32 stores orbitals in
// FP32 and runs H psi, the preconditioner and the rotations in FP32, while
// Gram matrices, residual norms, Cholesky, Rayleigh-Ritz and eigenvalues are
// FP64 (exact products with compensated accumulation, see linalg.cu).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "device.h"
#include "ham.h"
#include "learned.h"
#include "linalg.h"
#include "precond.h"
#include "solver_view.h"
#include "umma.h"

using namespace rs;

namespace rs {

// out[k] += sum_p A[p][k] B[p][k] for k < ncols (out zeroed by the caller),
// accumulated to FP64-level accuracy
template <typename T>
__global__ void k_coldots(const T *__restrict__ A, int64_t lda, const T *__restrict__ B, int64_t ldb, int ncols,
                          int64_t npts, double *out) {
    __shared__ double red[256];
    const int rows = blockDim.x / ncols;
    const int k = threadIdx.x % ncols, r = threadIdx.x / ncols;
    double acc = 0.0;
    if (r < rows) {
        if constexpr (sizeof(T) == 4) {
            // FP32 data on the FP32 pipes: every product split exactly
            // (p + pe = a b) and summed as an unevaluated pair (hi, lo) with
            // error-free additions, i.e. FP64-level accuracy
            float hi = 0.f, lo = 0.f;
            for (int64_t p = (int64_t)blockIdx.x * rows + r; p < npts; p += (int64_t)gridDim.x * rows) {
                const float a = A[p * lda + k], b = B[p * ldb + k];
                const float pr = __fmul_rn(a, b);   // _rn: never contracted
                const float pe = fmaf(a, b, -pr);
                const float sum = __fadd_rn(hi, pr);
                const float bb = __fsub_rn(sum, hi);
                const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(pr, bb));
                hi = sum;
                lo = __fadd_rn(lo, __fadd_rn(err, pe));
            }
            acc = (double)hi + (double)lo;
        } else {
            double comp = 0.0;  // Kahan-compensated FP64 sum of exact products
            for (int64_t p = (int64_t)blockIdx.x * rows + r; p < npts; p += (int64_t)gridDim.x * rows) {
                const double v = (double)A[p * lda + k] * (double)B[p * ldb + k];
                const double y = v - comp;
                const double t = acc + y;
                comp = (t - acc) - y;
                acc = t;
            }
        }
    }
    red[threadIdx.x] = r < rows ? acc : 0.0;
    __syncthreads();
    if (r == 0) {
        double s = 0;
        for (int q = 0; q < rows; ++q) s += red[q * ncols + k];
        atomicAdd(out + k, s);
    }
}

// Elementwise kernels over [npts][ncols] column blocks (ncols <= 256): a
// thread keeps one column k = tid % ncols, derives its per-column factor once
// and strides over rows, so no per-element index division or FP64 divide.
template <typename T>
__global__ void k_residual(const T *__restrict__ X, int64_t ldx, const T *__restrict__ HX, int64_t ldh,
                           const double *__restrict__ num, const double *__restrict__ den, T *__restrict__ R,
                           int64_t ldr, int ncols, int64_t npts) {
    const int rows = blockDim.x / ncols, k = threadIdx.x % ncols, r = threadIdx.x / ncols;
    if (r >= rows) return;
    const T lam = (T)(num[k] / den[k]);
    for (int64_t p = blockIdx.x * (int64_t)rows + r; p < npts; p += (int64_t)gridDim.x * rows)
        R[p * ldr + k] = HX[p * ldh + k] - lam * X[p * ldx + k];
}

__global__ void k_resnorm(const double *rr, int n, double dV, double *res) {
    const int k = threadIdx.x;
    if (k < n) res[k] = sqrt(dV * rr[k]);
}

template <typename T>
__global__ void k_scale_cols(T *Y, int64_t ldy, int ncols, int64_t npts, const double *nrm2, double dV) {
    const int rows = blockDim.x / ncols, k = threadIdx.x % ncols, r = threadIdx.x / ncols;
    if (r >= rows) return;
    const double n2 = dV * nrm2[k];
    if (!(n2 > 0)) return;
    const T f = (T)(1.0 / sqrt(n2));
    for (int64_t p = blockIdx.x * (int64_t)rows + r; p < npts; p += (int64_t)gridDim.x * rows) Y[p * ldy + k] *= f;
}

template <typename T>
__global__ void k_copy_cols(const T *__restrict__ S, int64_t lds, T *__restrict__ D, int64_t ldd, int ncols,
                            int64_t npts) {
    const int rows = blockDim.x / ncols, k = threadIdx.x % ncols, r = threadIdx.x / ncols;
    if (r >= rows) return;
    for (int64_t p = blockIdx.x * (int64_t)rows + r; p < npts; p += (int64_t)gridDim.x * rows)
        D[p * ldd + k] = S[p * lds + k];
}

__global__ void k_copy_leading(const double *A, int lda, int n, double *B, int ldb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x)
        B[(e / n) * ldb + e % n] = A[(e / n) * lda + e % n];
}

int coldots(int dtype, const void *A, int64_t lda, const void *B, int64_t ldb, int ncols, int64_t npts, double *out,
            cudaStream_t st) {
    RS_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * ncols, st));
    const int rows = 256 / ncols;
    const int64_t need = (npts + rows - 1) / rows;
    const unsigned blocks = (unsigned)std::min<int64_t>(need, 152 * 8);
    if (dtype == RS_F64)
        k_coldots<double><<<blocks, 256, 0, st>>>((const double *)A, lda, (const double *)B, ldb, ncols, npts, out);
    else
        k_coldots<float><<<blocks, 256, 0, st>>>((const float *)A, lda, (const float *)B, ldb, ncols, npts, out);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// ------------------------------------------------------------ RMM-DIIS ---
// Column-wise kernels over [npts][nb] blocks (ld = nb) for the RMM-DIIS
// refinement of every state (see rmm_block_step).

constexpr int RMM_MAXK = 9;       // iterates kept per state (n_steps + 1 <= 9)
constexpr int MD_MAX = 2 * RMM_MAXK;   // dot pairs of one k_multidot pass

struct DotPairs {
    const void *a[MD_MAX];
    const void *b[MD_MAX];
    int n;
};

// out[q * 64 + k] = sum_p a_q[p][k] b_q[p][k] for q < d.n, k < ncols (out
// zeroed by the caller), accumulated to FP64-level accuracy as in k_coldots.
// The pairs name their operands in a list of distinct arrays (d.arr, d.ia,
// d.ib): every array is read once per point row into the thread's own slots
// of shared memory and each pair takes its operands from there, so pairs
// that share an array do not read it from memory again.  Each pair's sum
// runs over the points in the same order as one pair alone would.
constexpr int MD_ARR = 2 * MD_MAX;
struct DotArrays {
    const void *arr[MD_ARR];
    unsigned char ia[MD_MAX], ib[MD_MAX];
    int narr, n;
};

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_multidot(DotArrays d, int ncols, int64_t npts, double *out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *vals = reinterpret_cast<T *>(smraw);   // [narr][blockDim]
    __shared__ double red[256];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int rows = nt / ncols;
    const int k = tid % ncols, r = tid / ncols;
    // compensated sums: FP32 (hi, lo) or FP64 (acc, comp) per pair
    T s0[NP], s1[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) s0[q] = s1[q] = T(0);
    if (r < rows) {
        for (int64_t p = (int64_t)blockIdx.x * rows + r; p < npts; p += (int64_t)gridDim.x * rows) {
            for (int j = 0; j < d.narr; ++j) vals[j * nt + tid] = ((const T *)d.arr[j])[p * ncols + k];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                if (q >= d.n) break;
                const T a = vals[d.ia[q] * nt + tid], b = vals[d.ib[q] * nt + tid];
                if constexpr (sizeof(T) == 4) {
                    const float pr = __fmul_rn(a, b);
                    const float pe = fmaf(a, b, -pr);
                    const float sum = __fadd_rn(s0[q], pr);
                    const float bb = __fsub_rn(sum, s0[q]);
                    const float err = __fadd_rn(__fsub_rn(s0[q], __fsub_rn(sum, bb)), __fsub_rn(pr, bb));
                    s0[q] = sum;
                    s1[q] = __fadd_rn(s1[q], __fadd_rn(err, pe));
                } else {
                    const double v = a * b;
                    const double y = v - s1[q];
                    const double t = s0[q] + y;
                    s1[q] = (t - s0[q]) - y;
                    s0[q] = t;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        if (q >= d.n) break;
        double acc = 0.0;
        if (r < rows) acc = sizeof(T) == 4 ? (double)s0[q] + (double)s1[q] : (double)s0[q];
        red[tid] = r < rows ? acc : 0.0;
        __syncthreads();
        if (r == 0) {
            double t = 0;
            for (int qq = 0; qq < rows; ++qq) t += red[qq * ncols + k];
            atomicAdd(out + q * 64 + k, t);
        }
        __syncthreads();
    }
}

// Lowest eigenpair of the symmetric pencil (A, B) of order n <= RMM_MAXK
// (row-major n x n): B = U^T U (Cholesky; false when a pivot^2 falls below
// 1e-12 of its diagonal), cyclic Jacobi on U^-T A U^-1, v = U^-1 y.
__device__ bool small_pencil_lowest(int n, const double *A, const double *B, double *v) {
    double U[RMM_MAXK][RMM_MAXK], Ui[RMM_MAXK][RMM_MAXK], C[RMM_MAXK][RMM_MAXK], V[RMM_MAXK][RMM_MAXK];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) U[i][j] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = 0.5 * (B[j * n + j] + B[j * n + j]);
        for (int k = 0; k < j; ++k) d -= U[k][j] * U[k][j];
        if (!(d > 1e-12 * B[j * n + j])) return false;
        const double ujj = sqrt(d);
        U[j][j] = ujj;
        for (int i = j + 1; i < n; ++i) {
            double t = 0.5 * (B[j * n + i] + B[i * n + j]);
            for (int k = 0; k < j; ++k) t -= U[k][j] * U[k][i];
            U[j][i] = t / ujj;
        }
    }
    for (int c = 0; c < n; ++c)
        for (int i = n - 1; i >= 0; --i) {
            double t = i == c ? 1.0 : 0.0;
            for (int k = i + 1; k < n; ++k) t -= U[i][k] * Ui[k][c];
            Ui[i][c] = i > c ? 0.0 : t / U[i][i];
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double t = 0;
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) t += Ui[a][i] * 0.5 * (A[a * n + b] + A[b * n + a]) * Ui[b][j];
            C[i][j] = t;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0, dia = 0;
        for (int i = 0; i < n; ++i) {
            dia += C[i][i] * C[i][i];
            for (int j = i + 1; j < n; ++j) off += C[i][j] * C[i][j];
        }
        if (off <= 1e-32 * dia) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (C[p][q] == 0.0) continue;
                const double th = (C[q][q] - C[p][p]) / (2.0 * C[p][q]);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double ckp = C[k][p], ckq = C[k][q];
                    C[k][p] = c * ckp - s * ckq;
                    C[k][q] = s * ckp + c * ckq;
                }
                for (int k = 0; k < n; ++k) {
                    const double cpk = C[p][k], cqk = C[q][k];
                    C[p][k] = c * cpk - s * cqk;
                    C[q][k] = s * cpk + c * cqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int lo = 0;
    for (int i = 1; i < n; ++i)
        if (C[i][i] < C[lo][lo]) lo = i;
    for (int i = 0; i < n; ++i) {
        double t = 0;
        for (int k = 0; k < n; ++k) t += Ui[i][k] * V[k][lo];
        v[i] = t;
    }
    return true;
}

// Trial step of every column: lambda minimising the Rayleigh quotient of
// x + lambda p, from the dots (xx, xp, pp, xhx, xhp, php) at rows q * 64;
// 0 for columns whose residual norm is <= tol (converged states stay).
__global__ void k_rmm_lambda(const double *dots, const double *res, double tol, int nb, double *lam) {
    const int k = threadIdx.x;
    if (k >= nb) return;
    double l = 0.0;
    if (res[k] > tol) {
        const double B[4] = {dots[0 * 64 + k], dots[1 * 64 + k], dots[1 * 64 + k], dots[2 * 64 + k]};
        const double A[4] = {dots[3 * 64 + k], dots[4 * 64 + k], dots[4 * 64 + k], dots[5 * 64 + k]};
        double v[2];
        if (small_pencil_lowest(2, A, B, v) && v[0] != 0.0) l = v[1] / v[0];
    }
    lam[k] = l;
}

// DIIS coefficients of every column over n iterates: the lowest pair of
// (A, B), A_ij = <r_i|r_j>, B_ij = <x_i|x_j> (stored [i][j][64]), alpha
// normalised to <xbar|xbar> = 1 and sum alpha >= 0; the latest iterate alone
// when the iterates are numerically dependent.  alpha out [i][64].
__global__ void k_rmm_diis(const double *A, const double *B, int n, int nb, double *alpha) {
    const int k = threadIdx.x;
    if (k >= nb) return;
    double a[RMM_MAXK * RMM_MAXK], b[RMM_MAXK * RMM_MAXK], v[RMM_MAXK];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            a[i * n + j] = A[(i * RMM_MAXK + j) * 64 + k];
            b[i * n + j] = B[(i * RMM_MAXK + j) * 64 + k];
        }
    if (small_pencil_lowest(n, a, b, v)) {
        double s = 0;
        for (int i = 0; i < n; ++i) s += v[i];
        const double sg = s >= 0 ? 1.0 : -1.0;
        for (int i = 0; i < n; ++i) alpha[i * 64 + k] = sg * v[i];
    } else {
        for (int i = 0; i < n; ++i) alpha[i * 64 + k] = i == n - 1 ? 1.0 : 0.0;
    }
}

// xbar = sum_i alpha_i x_i, likewise H x and r, over n iterates stored at
// hist + i * stride (x), + (slots + i) * stride (Hx), + (2 slots + i) * stride (r)
template <typename T>
__global__ void k_rmm_combine(const T *__restrict__ hist, int64_t stride, int slots, int n,
                              const double *__restrict__ alpha, int nb, int64_t npts, T *__restrict__ xb,
                              T *__restrict__ hxb, T *__restrict__ rb) {
    const int rows = blockDim.x / nb, k = threadIdx.x % nb, r = threadIdx.x / nb;
    if (r >= rows) return;
    T al[RMM_MAXK];
    for (int i = 0; i < RMM_MAXK; ++i) al[i] = i < n ? (T)alpha[i * 64 + k] : T(0);
    for (int64_t p = blockIdx.x * (int64_t)rows + r; p < npts; p += (int64_t)gridDim.x * rows) {
        const int64_t e = p * nb + k;
        T x = 0, hx = 0, rr = 0;
        for (int i = 0; i < n; ++i) {
            x += al[i] * hist[i * stride + e];
            hx += al[i] * hist[(slots + i) * stride + e];
            rr += al[i] * hist[(2 * slots + i) * stride + e];
        }
        xb[e] = x;
        hxb[e] = hx;
        rb[e] = rr;
    }
}

// x_out = x + lambda p, hx_out = hx + lambda hp (per-column lambda)
template <typename T>
__global__ void k_rmm_step(const T *__restrict__ x, const T *__restrict__ hx, const T *__restrict__ pp,
                           const T *__restrict__ hp, const double *__restrict__ lam, int nb, int64_t npts,
                           T *__restrict__ xo, T *__restrict__ hxo) {
    const int rows = blockDim.x / nb, k = threadIdx.x % nb, r = threadIdx.x / nb;
    if (r >= rows) return;
    const T l = (T)lam[k];
    for (int64_t p = blockIdx.x * (int64_t)rows + r; p < npts; p += (int64_t)gridDim.x * rows) {
        const int64_t e = p * nb + k;
        xo[e] = x[e] + l * pp[e];
        hxo[e] = hx[e] + l * hp[e];
    }
}

// A / B of the DIIS pencil from a k_multidot pass: pair q holds <r_i|r_j>
// (kind 0) or <x_i|x_j> (kind 1) for (i, j) = idx[q]; stored symmetric.
struct PairIndex {
    int kind[MD_MAX], i[MD_MAX], j[MD_MAX], n;
};
__global__ void k_rmm_store(const double *dots, PairIndex t, int nb, double *A, double *B) {
    const int k = threadIdx.x;
    if (k >= nb) return;
    for (int q = 0; q < t.n; ++q) {
        double *M = t.kind[q] == 0 ? A : B;
        const double v = dots[q * 64 + k];
        M[(t.i[q] * RMM_MAXK + t.j[q]) * 64 + k] = v;
        M[(t.j[q] * RMM_MAXK + t.i[q]) * 64 + k] = v;
    }
}

int multidot(int dtype, const DotPairs &d, int ncols, int64_t npts, double *out, cudaStream_t st) {
    if (d.n < 1 || d.n > MD_MAX) return fail(RS_EINVAL, "multidot: %d pairs", d.n);
    RS_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 64 * d.n, st));
    // the distinct operand arrays of the pairs
    DotArrays a{};
    auto slot = [&](const void *ptr) {
        for (int j = 0; j < a.narr; ++j)
            if (a.arr[j] == ptr) return j;
        a.arr[a.narr] = ptr;
        return a.narr++;
    };
    for (int q = 0; q < d.n; ++q) {
        a.ia[q] = (unsigned char)slot(d.a[q]);
        a.ib[q] = (unsigned char)slot(d.b[q]);
    }
    a.n = d.n;
    const int rows = 256 / ncols;
    const unsigned blocks = (unsigned)std::min<int64_t>((npts + rows - 1) / rows, 152 * 8);
    const size_t es = dtype == RS_F64 ? 8 : 4, smem = (size_t)a.narr * 256 * es;
    // the usual passes hold at most six pairs: a kernel with registers for
    // six sums keeps more warps resident than one sized for MD_MAX
    auto launch = [&](const void *fn, auto kern) -> int {
        RS_TRY(smem_optin(fn, smem));
        kern<<<blocks, 256, smem, st>>>(a, ncols, npts, out);
        return RS_OK;
    };
    if (dtype == RS_F64) {
        if (d.n <= 6) RS_TRY(launch((const void *)k_multidot<double, 6>, k_multidot<double, 6>));
        else RS_TRY(launch((const void *)k_multidot<double, MD_MAX>, k_multidot<double, MD_MAX>));
    } else {
        if (d.n <= 6) RS_TRY(launch((const void *)k_multidot<float, 6>, k_multidot<float, 6>));
        else RS_TRY(launch((const void *)k_multidot<float, MD_MAX>, k_multidot<float, MD_MAX>));
    }
    RS_LAUNCH_CHECK();
    return RS_OK;
}

}  // namespace rs

struct rs_solver {
    rs_ham *h = nullptr;
    rs_solver_cfg cfg{};
    int64_t npts = 0;
    double dV = 0;
    int es = 8;
    int nblk = 0;
    DevBuf psi, hpsi, P, Z, HZ, R, small, la, eig, res, tcbuf, psi64, hpsi64, rr64, gs_tbuf, gs_nbuf;
    TcWork tc;
    UmmaSplitCache gs_t, gs_n;   // FP32 mode: splits of Psi[:, :(b+1) nb] within a block step
    std::vector<char> has_p;
    Precond *pc = nullptr;
    // learned preconditioner: the FP32 weights last set or trained
    DevBuf wlearn;
    bool has_wlearn = false;
    // schedules and statistics (rs_solver_stats)
    int sweeps = 0, eps_f64 = 0, fallback_sweep = 0, stall = 0;
    double best = std::numeric_limits<double>::infinity(), max_res = 0;
    double train_target_s = 0, train_fit_s = 0;
    double lam_max = 0;   // power-iteration estimate of the largest eigenvalue of H (0: not taken)
    DevBuf eps64;   // FP64 Rayleigh-Ritz eigenvalues when the caller passes no eps_dev
    // RMM-DIIS: iterates x_i, H x_i, r_i ([slot][npts][nb] each kind), p, H p,
    // the combinations, and the small per-column arrays
    DevBuf rmm_hist, rmm_small;
    int rmm_M = 3;
    // small FP64 buffers (inside `small`)
    double *dots = nullptr, *M = nullptr, *G = nullptr, *A = nullptr, *U = nullptr, *Ui = nullptr, *T1 = nullptr,
           *At = nullptr, *Yv = nullptr, *mu = nullptr, *C = nullptr;
    int *status = nullptr;
    void *eighw = nullptr;
    ~rs_solver() { delete pc; }
};

namespace {

// grid of the column-block kernels (256 threads, 256 / ncols rows per CTA pass)
unsigned elem_blocks(int64_t npts, int ncols) {
    const int64_t rows = std::max(1, 256 / ncols);
    return (unsigned)std::min<int64_t>((npts + rows - 1) / rows, 152 * 16);
}

int copy_cols(int dtype, const void *S, int64_t lds, void *D, int64_t ldd, int ncols, int64_t npts, cudaStream_t st) {
    if (dtype == RS_F64)
        k_copy_cols<double><<<elem_blocks(npts, ncols), 256, 0, st>>>((const double *)S, lds, (double *)D, ldd, ncols, npts);
    else
        k_copy_cols<float><<<elem_blocks(npts, ncols), 256, 0, st>>>((const float *)S, lds, (float *)D, ldd, ncols, npts);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// inner-iteration contractions: FP32 mode on the tensor cores (FP32-level
// accuracy), FP64 mode on the FP64 pipes
int gram_any(int dtype, const void *X, int64_t ldx, int nx, const void *Y, int64_t ldy, int ny, int64_t npts, double dV,
             double *S, int64_t lds, cudaStream_t st, const TcWork &tc, UmmaSplitCache *xcache = nullptr) {
    if (dtype == RS_F64)
        return gram<double>((const double *)X, ldx, nx, (const double *)Y, ldy, ny, npts, dV, S, lds, st);
    if (tc.p && tc.bytes >= umma_work_bytes(nx, ny, npts))
        return umma_gram((const float *)X, ldx, nx, (const float *)Y, ldy, ny, npts, dV, S, lds, tc.p, tc.err, st,
                         xcache);
    return gram<float>((const float *)X, ldx, nx, (const float *)Y, ldy, ny, npts, dV, S, lds, st, true);
}

int rowmul_any(int dtype, const void *X, int64_t ldx, int n, const double *C, int64_t ldc, int m, void *Y, int64_t ldy,
               int64_t npts, double alpha, double beta, cudaStream_t st, const TcWork &tc,
               UmmaSplitCache *xcache = nullptr) {
    if (dtype == RS_F64)
        return rowmul<double>((const double *)X, ldx, n, C, ldc, m, (double *)Y, ldy, npts, alpha, beta, st);
    if (tc.p && tc.bytes >= umma_work_bytes(npts, m, n))
        return umma_rowmul((const float *)X, ldx, n, C, ldc, m, (float *)Y, ldy, npts, alpha, beta, tc.p, tc.err, st,
                           xcache);
    return rowmul<float>((const float *)X, ldx, n, C, ldc, m, (float *)Y, ldy, npts, alpha, beta, st);
}

const char *off(const DevBuf &b, int64_t elems, int es) { return (const char *)b.p + (size_t)elems * es; }
char *offw(DevBuf &b, int64_t elems, int es) { return (char *)b.p + (size_t)elems * es; }

// One LOBPCG update of block b.  Blocking (reads the block's residuals and
// the Cholesky status).
int block_step(rs_solver *S, int b, cudaStream_t st) {
    const rs_solver_cfg &c = S->cfg;
    const int nb = c.nb, nst = c.nst, dt = c.dtype, es = S->es;
    const int64_t np = S->npts;
    const int64_t ldz = 3 * nb;
    const void *X = off(S->psi, (int64_t)b * nb, es);
    const void *HX = off(S->hpsi, (int64_t)b * nb, es);
    double *num = S->dots, *den = S->dots + 64, *rr = S->dots + 128, *nrm = S->dots + 256;
    // 1. Rayleigh quotients, residuals and their norms
    RS_TRY(coldots(dt, X, nst, HX, nst, nb, np, num, st));
    RS_TRY(coldots(dt, X, nst, X, nst, nb, np, den, st));
    if (dt == RS_F64)
        k_residual<double><<<elem_blocks(np, nb), 256, 0, st>>>((const double *)X, nst, (const double *)HX, nst, num,
                                                                den, S->R.as<double>(), nb, nb, np);
    else
        k_residual<float><<<elem_blocks(np, nb), 256, 0, st>>>((const float *)X, nst, (const float *)HX, nst, num, den,
                                                               S->R.as<float>(), nb, nb, np);
    RS_LAUNCH_CHECK();
    RS_TRY(coldots(dt, S->R.p, nb, S->R.p, nb, nb, np, rr, st));
    double *resb = S->res.as<double>() + (size_t)b * nb;
    k_resnorm<<<1, 64, 0, st>>>(rr, nb, S->dV, resb);
    RS_LAUNCH_CHECK();
    std::vector<double> res(nb);
    RS_CUDA(cudaMemcpyAsync(res.data(), resb, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    // a bounded wait of an earlier H psi launch that gave up leaves incomplete
    // data behind: stop before it spreads into the residuals
    int ringerr = 0;
    if (int *rw = ham_status_word(S->h)) RS_CUDA(cudaMemcpyAsync(&ringerr, rw, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    if (ringerr) return fail(RS_ETIMEOUT, "eigensolver: an H psi pipeline wait timed out");
    bool conv = true;
    for (double r : res) {
        if (!std::isfinite(r)) return fail(RS_ENAN, "eigensolver: non-finite residual in block %d", b);
        conv = conv && r <= c.tol;
    }
    if (conv) return RS_OK;

    // 2. W = K R into Z[:, nb:2nb]; X, P_b, HX into Z / HZ
    RS_TRY(S->pc->apply(S->h, S->R.p, nb, offw(S->Z, nb, es), ldz, nb, dt, st));
    RS_TRY(copy_cols(dt, X, nst, S->Z.p, ldz, nb, np, st));
    RS_TRY(copy_cols(dt, HX, nst, S->HZ.p, ldz, nb, np, st));
    const bool use_p = S->has_p[b] != 0;
    if (use_p) RS_TRY(copy_cols(dt, off(S->P, (int64_t)b * nb, es), nst, offw(S->Z, 2 * nb, es), ldz, nb, np, st));
    const int ny = use_p ? 2 * nb : nb;
    void *Y = offw(S->Z, nb, es);

    // 3. classical Gram-Schmidt, twice, against Psi[:, :(b+1) nb]
    // (Psi does not change between the passes: its two BF16x3 splits, one per
    // contraction layout, are made in the first pass and reused in the second)
    const int nq = (b + 1) * nb;
    S->gs_t.valid = S->gs_n.valid = false;
    for (int pass = 0; pass < 2; ++pass) {
        RS_TRY(gram_any(dt, S->psi.p, nst, nq, Y, ldz, ny, np, S->dV, S->M, ny, st, S->tc, &S->gs_t));
        RS_TRY(rowmul_any(dt, S->psi.p, nst, nq, S->M, ny, ny, Y, ldz, np, -1.0, 1.0, st, S->tc, &S->gs_n));
    }
    RS_TRY(coldots(dt, Y, ldz, Y, ldz, ny, np, nrm, st));
    if (dt == RS_F64)
        k_scale_cols<double><<<elem_blocks(np, ny), 256, 0, st>>>((double *)Y, ldz, ny, np, nrm, S->dV);
    else
        k_scale_cols<float><<<elem_blocks(np, ny), 256, 0, st>>>((float *)Y, ldz, ny, np, nrm, S->dV);
    RS_LAUNCH_CHECK();

    // 4. H Y
    RS_TRY(rs_ham_apply_block(S->h, Y, ldz, offw(S->HZ, nb, es), ldz, nb, dt, st));
    if (use_p) RS_TRY(rs_ham_apply_block(S->h, offw(S->Z, 2 * nb, es), ldz, offw(S->HZ, 2 * nb, es), ldz, nb, dt, st));

    // 5. Rayleigh-Ritz on Z = [X, Y]
    int n = nb + ny;
    RS_TRY(gram_any(dt, S->Z.p, ldz, n, S->Z.p, ldz, n, np, S->dV, S->G, n, st, S->tc));
    RS_TRY(gram_any(dt, S->Z.p, ldz, n, S->HZ.p, ldz, n, np, S->dV, S->A, n, st, S->tc));
    RS_TRY(symmetrize(S->G, n, n, st));
    RS_TRY(symmetrize(S->A, n, n, st));
    int bad = 1;
    for (int attempt = 0; attempt < 2 && bad; ++attempt) {
        if (attempt == 1) {
            if (n == 2 * nb) break;
            n = 2 * nb;  // drop P
        }
        k_copy_leading<<<64, 256, 0, st>>>(S->G, nb + ny, n, S->U, n);
        RS_LAUNCH_CHECK();
        // a pivot below what the Gram matrix's own accuracy resolves means the
        // search space is numerically dependent (FP32 mode: FP32-accumulated G)
        RS_TRY(cholesky(S->U, n, n, dt == RS_F32 ? 1e-5 : 1e-12, S->status, st));
        RS_CUDA(cudaMemcpyAsync(&bad, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
    }
    if (bad) return RS_OK;  // no usable search space this sweep; the block keeps X
    const int lda = nb + ny;
    RS_TRY(tri_inv(S->U, n, n, S->Ui, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, S->Ui, n, true, S->A, lda, false, 0.0, S->T1, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, S->T1, n, false, S->Ui, n, false, 0.0, S->At, n, st));
    RS_TRY(symmetrize(S->At, n, n, st));
    // inner Rayleigh-Ritz: FP32 Jacobi is enough in FP32 mode; FP64 mode refines
    RS_TRY(eigh(S->At, n, n, S->mu, S->Yv, n, dt == RS_F32 ? -1 : 2, S->status, S->eighw, st));
    RS_TRY(gemm_small(n, nb, n, 1.0, S->Ui, n, false, S->Yv, n, false, 0.0, S->C, nb, st));

    // 6. X <- Z C, P <- Z[:, nb:n] C[nb:n, :]
    RS_TRY(rowmul_any(dt, S->Z.p, ldz, n, S->C, nb, nb, offw(S->psi, (int64_t)b * nb, es), nst, np, 1.0, 0.0, st, S->tc));
    RS_TRY(rowmul_any(dt, offw(S->Z, nb, es), ldz, n - nb, S->C + (size_t)nb * nb, nb, nb,
                      offw(S->P, (int64_t)b * nb, es), nst, np, 1.0, 0.0, st, S->tc));
    S->has_p[b] = 1;
    return RS_OK;
}

// One RMM-DIIS refinement of block b (the paper's eigensolver, Sec. III:
// Wood and Zunger 1985, Kresse and Furthmueller 1996), every state on its own:
//   x_0 = psi, e_i = <x_i|H x_i>/<x_i|x_i>, r_i = H x_i - e_i x_i; a block whose
//   states all have ||r_0|| <= tol is left alone (Sec. VIII);
//   p = K r_0, lambda minimises the Rayleigh quotient of x_0 + lambda p,
//   x_1 = x_0 + lambda p;
//   then n_steps - 1 DIIS steps: alpha = the lowest pair of the pencil
//   (<r_i|r_j>, <x_i|x_j>), xbar = sum alpha_i x_i, rbar = sum alpha_i r_i,
//   x_{m+1} = xbar + lambda K rbar;  psi <- x_{n_steps}.
// H is applied once per step (H x_{m+1} = H xbar + lambda H p).  Blocking
// (reads the block's residuals).
int rmm_block_step(rs_solver *S, int b, cudaStream_t st) {
    const rs_solver_cfg &c = S->cfg;
    const int nb = c.nb, nst = c.nst, dt = c.dtype, es = S->es, M = S->rmm_M, slots = M + 1;
    const int64_t np = S->npts, sz = np * nb;
    char *hist = (char *)S->rmm_hist.p;
    auto X = [&](int i) { return (void *)(hist + (size_t)i * sz * es); };
    auto HX = [&](int i) { return (void *)(hist + (size_t)(slots + i) * sz * es); };
    auto R = [&](int i) { return (void *)(hist + (size_t)(2 * slots + i) * sz * es); };
    void *P = hist + (size_t)(3 * slots) * sz * es, *HP = hist + (size_t)(3 * slots + 1) * sz * es;
    void *XB = hist + (size_t)(3 * slots + 2) * sz * es, *HXB = hist + (size_t)(3 * slots + 3) * sz * es;
    void *RB = hist + (size_t)(3 * slots + 4) * sz * es;
    double *dots = S->rmm_small.as<double>();            // [MD_MAX][64]
    double *A = dots + MD_MAX * 64, *B = A + RMM_MAXK * RMM_MAXK * 64;
    double *alpha = B + RMM_MAXK * RMM_MAXK * 64, *lam = alpha + RMM_MAXK * 64;
    double *rr = lam + 64;
    const unsigned eb = elem_blocks(np, nb);
    auto residual = [&](int i) -> int {   // e_i and r_i of iterate i
        DotPairs d{};
        d.a[0] = X(i), d.b[0] = HX(i), d.a[1] = X(i), d.b[1] = X(i), d.n = 2;
        RS_TRY(multidot(dt, d, nb, np, dots, st));
        if (dt == RS_F64)
            k_residual<double><<<eb, 256, 0, st>>>((const double *)X(i), nb, (const double *)HX(i), nb, dots, dots + 64,
                                                   (double *)R(i), nb, nb, np);
        else
            k_residual<float><<<eb, 256, 0, st>>>((const float *)X(i), nb, (const float *)HX(i), nb, dots, dots + 64,
                                                  (float *)R(i), nb, nb, np);
        RS_LAUNCH_CHECK();
        return RS_OK;
    };
    RS_TRY(copy_cols(dt, off(S->psi, (int64_t)b * nb, es), nst, X(0), nb, nb, np, st));
    RS_TRY(copy_cols(dt, off(S->hpsi, (int64_t)b * nb, es), nst, HX(0), nb, nb, np, st));
    RS_TRY(residual(0));
    RS_TRY(coldots(dt, R(0), nb, R(0), nb, nb, np, rr, st));
    double *resb = S->res.as<double>() + (size_t)b * nb;
    k_resnorm<<<1, 64, 0, st>>>(rr, nb, S->dV, resb);
    RS_LAUNCH_CHECK();
    std::vector<double> res(nb);
    RS_CUDA(cudaMemcpyAsync(res.data(), resb, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    int ringerr = 0;
    if (int *rw = ham_status_word(S->h)) RS_CUDA(cudaMemcpyAsync(&ringerr, rw, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    if (ringerr) return fail(RS_ETIMEOUT, "eigensolver: an H psi pipeline wait timed out");
    bool conv = true;
    for (double r : res) {
        if (!std::isfinite(r)) return fail(RS_ENAN, "eigensolver: non-finite residual in block %d", b);
        conv = conv && r <= c.tol;
    }
    if (conv) return RS_OK;
    // step 0: the Rayleigh-quotient trial step along p = K r_0
    RS_TRY(S->pc->apply(S->h, R(0), nb, P, nb, nb, dt, st));
    RS_TRY(rs_ham_apply_block(S->h, P, nb, HP, nb, nb, dt, st));
    {
        DotPairs d{};
        const void *a[6] = {X(0), X(0), P, X(0), X(0), P}, *bb[6] = {X(0), P, P, HX(0), HP, HP};
        for (int q = 0; q < 6; ++q) d.a[q] = a[q], d.b[q] = bb[q];
        d.n = 6;
        RS_TRY(multidot(dt, d, nb, np, dots, st));
        k_rmm_lambda<<<1, 64, 0, st>>>(dots, resb, c.tol, nb, lam);
        RS_LAUNCH_CHECK();
    }
    auto advance = [&](const void *x, const void *hx, int to) -> int {
        if (dt == RS_F64)
            k_rmm_step<double><<<eb, 256, 0, st>>>((const double *)x, (const double *)hx, (const double *)P,
                                                   (const double *)HP, lam, nb, np, (double *)X(to), (double *)HX(to));
        else
            k_rmm_step<float><<<eb, 256, 0, st>>>((const float *)x, (const float *)hx, (const float *)P,
                                                  (const float *)HP, lam, nb, np, (float *)X(to), (float *)HX(to));
        RS_LAUNCH_CHECK();
        return RS_OK;
    };
    RS_TRY(advance(X(0), HX(0), 1));
    for (int m = 1; m < M; ++m) {
        RS_TRY(residual(m));
        // column m of the DIIS pencil (and column 0 at the first DIIS step)
        DotPairs d{};
        PairIndex t{};
        for (int col = (m == 1 ? 0 : m); col <= m; ++col)
            for (int i = 0; i <= col; ++i)
                for (int kind = 0; kind < 2; ++kind) {
                    d.a[d.n] = kind == 0 ? R(i) : X(i);
                    d.b[d.n] = kind == 0 ? R(col) : X(col);
                    t.kind[t.n] = kind, t.i[t.n] = i, t.j[t.n] = col;
                    ++d.n, ++t.n;
                }
        RS_TRY(multidot(dt, d, nb, np, dots, st));
        k_rmm_store<<<1, 64, 0, st>>>(dots, t, nb, A, B);
        k_rmm_diis<<<1, 64, 0, st>>>(A, B, m + 1, nb, alpha);
        RS_LAUNCH_CHECK();
        if (dt == RS_F64)
            k_rmm_combine<double><<<eb, 256, 0, st>>>((const double *)hist, sz, slots, m + 1, alpha, nb, np,
                                                      (double *)XB, (double *)HXB, (double *)RB);
        else
            k_rmm_combine<float><<<eb, 256, 0, st>>>((const float *)hist, sz, slots, m + 1, alpha, nb, np,
                                                     (float *)XB, (float *)HXB, (float *)RB);
        RS_LAUNCH_CHECK();
        RS_TRY(S->pc->apply(S->h, RB, nb, P, nb, nb, dt, st));
        RS_TRY(rs_ham_apply_block(S->h, P, nb, HP, nb, nb, dt, st));
        RS_TRY(advance(XB, HXB, m + 1));
    }
    return copy_cols(dt, X(M), nb, offw(S->psi, (int64_t)b * nb, es), nst, nb, np, st);
}

}  // namespace

__global__ void k_widen(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = (double)a[e];
}

static int rayleigh_ritz_f64_impl(rs_solver *S, double *eps_dev, cudaStream_t st) {
    const rs_solver_cfg &c = S->cfg;
    const int n = c.nst;
    if (c.dtype == RS_F64) {
        RS_CUDA(cudaMemcpyAsync(eps_dev, S->eig.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        RS_CUDA(cudaStreamSynchronize(st));
        return RS_OK;
    }
    const size_t nn = (size_t)n * n;
    if (!S->psi64.p) {
        RS_TRY(S->psi64.alloc(sizeof(double) * (size_t)S->npts * n));
        RS_TRY(S->hpsi64.alloc(sizeof(double) * (size_t)S->npts * n));
        RS_TRY(S->rr64.alloc(sizeof(double) * (4 * nn + 16) + eigh_work_bytes(n)));
    }
    double *Sm = S->rr64.as<double>(), *h = Sm + nn, *Ui = h + nn, *T = Ui + nn;
    int *status = reinterpret_cast<int *>(T + nn);
    void *ew = reinterpret_cast<void *>(T + nn + 16);
    // FP64 copy of the FP32 orbitals, H applied in FP64
    k_widen<<<1024, 256, 0, st>>>(S->psi.as<float>(), S->psi64.as<double>(), S->npts * n);
    RS_LAUNCH_CHECK();
    for (int b = 0; b < n; b += c.nb)
        RS_TRY(rs_ham_apply_block(S->h, S->psi64.as<double>() + b, n, S->hpsi64.as<double>() + b, n, c.nb, RS_F64, st));
    // generalized Rayleigh-Ritz h x = eps S x with S, h accumulated in FP64
    // (the overlap of the FP32 orbitals is exact: products of FP32 values)
    RS_TRY(gram<float>(S->psi.as<float>(), n, n, S->psi.as<float>(), n, n, S->npts, S->dV, Sm, n, st));
    RS_TRY(gram<double>(S->psi64.as<double>(), n, n, S->hpsi64.as<double>(), n, n, S->npts, S->dV, h, n, st));
    RS_TRY(symmetrize(Sm, n, n, st));
    RS_TRY(symmetrize(h, n, n, st));
    RS_TRY(cholesky(Sm, n, n, 1e-14, status, st));
    RS_TRY(tri_inv(Sm, n, n, Ui, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, Ui, n, true, h, n, false, 0.0, T, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, T, n, false, Ui, n, false, 0.0, h, n, st));
    RS_TRY(symmetrize(h, n, n, st));
    RS_TRY(eigh(h, n, n, eps_dev, T, n, 2, status, ew, st));
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

// out[k] = sum_p (Q[p][k] - eps[k] P[p][k])^2, Kahan-compensated FP64 sums;
// grid (column chunks of 256, row chunks), out zeroed by the caller
__global__ void k_resid_norm2(const double *__restrict__ P, const double *__restrict__ Q, int64_t ld, int n,
                              const double *__restrict__ eps, int64_t npts, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double e = eps[k];
    double acc = 0, comp = 0;
    for (int64_t p = blockIdx.y; p < npts; p += gridDim.y) {
        const double d = Q[p * ld + k] - e * P[p * ld + k];
        const double y = d * d - comp;
        const double t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    }
    atomicAdd(out + k, acc);
}

__global__ void k_sqrt_scale(double *a, int n, double s) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) a[k] = sqrt(s * a[k]);
}

// one damped Richardson step per column, P[p][k] -= (Q[p][k] - eps[k] P[p][k]) / (lam - eps[k])
__global__ void k_smooth_step(double *__restrict__ P, const double *__restrict__ Q, const double *__restrict__ eps,
                              double lam, int n, int64_t total) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % n);
        const double t = eps[k];
        P[e] -= (Q[e] - t * P[e]) / (lam - t);
    }
}

// power iteration: a fixed pseudo-random start vector (splitmix64 of the index)
__global__ void k_pi_start(double *x, int64_t npts) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)p + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[p] = (double)(z >> 11) * 0x1.0p-53 - 0.5;
    }
}

// acc[0] += sum x y', acc[1] += sum y'^2 with y' = y - sigma x (one CTA per chunk)
__global__ void k_pi_dots(const double *__restrict__ x, const double *__restrict__ y, double sigma, int64_t npts,
                          double *acc) {
    __shared__ double red[2][32];
    double a = 0, b = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x) {
        const double v = y[p] - sigma * x[p];
        a += x[p] * v;
        b += v * v;
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!lane) {
        red[0][wid] = a;
        red[1][wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? red[0][lane] : 0;
        b = lane < nw ? red[1][lane] : 0;
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (!lane) {
            atomicAdd(acc, a);
            atomicAdd(acc + 1, b);
        }
    }
}

// x <- (y - sigma x) / ||y - sigma x|| (acc[1] holds the squared norm;
// every iteration accumulates into its own pair of zeroed words)
__global__ void k_pi_scale(double *__restrict__ x, const double *__restrict__ y, double sigma, int64_t npts,
                           const double *acc) {
    const double s = acc[1] > 0 ? 1.0 / sqrt(acc[1]) : 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x)
        x[p] = (y[p] - sigma * x[p]) * s;
}

// largest eigenvalue of H: power iteration on H - sigma with sigma the
// solver's lowest Ritz value (an upper bound of the lowest eigenvalue, so
// that H - sigma is positive up to that small overlap and the iteration
// converges to the top of the spectrum), Rayleigh quotient of the last
// iterate.  A Rayleigh quotient never exceeds lambda_max.
static int lambda_max_estimate(rs_solver *S, double *x, double *y, cudaStream_t st, double *out) {
    constexpr int ITERS = 120;
    double sigma = 0;
    RS_CUDA(cudaMemcpyAsync(&sigma, S->eig.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    DevBuf acc;
    RS_TRY(acc.alloc(sizeof(double) * 2 * (ITERS + 1)));
    RS_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(double) * 2 * (ITERS + 1), st));
    const int64_t n = S->npts;
    const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_pi_start<<<g, 256, 0, st>>>(x, n);
    k_pi_dots<<<g, 256, 0, st>>>(x, x, 0.0, n, acc.as<double>());
    k_pi_scale<<<g, 256, 0, st>>>(x, x, 0.0, n, acc.as<double>());
    RS_LAUNCH_CHECK();
    for (int it = 1; it <= ITERS; ++it) {
        double *a = acc.as<double>() + 2 * it;
        RS_TRY(rs_ham_apply_block(S->h, x, 1, y, 1, 1, RS_F64, st));
        k_pi_dots<<<g, 256, 0, st>>>(x, y, sigma, n, a);
        if (it < ITERS) k_pi_scale<<<g, 256, 0, st>>>(x, y, sigma, n, a);
        RS_LAUNCH_CHECK();
    }
    double last[2] = {0, 0};
    RS_CUDA(cudaMemcpyAsync(last, acc.as<double>() + 2 * ITERS, sizeof(last), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    // x has unit norm: the Rayleigh quotient of H - sigma is x . (H - sigma) x
    if (!std::isfinite(last[0]) || !(last[0] > 0)) return fail(RS_ENAN, "lambda_max estimate failed");
    *out = last[0] + sigma;
    return RS_OK;
}

static int certify_impl(rs_solver *S, int n_smooth, double lam, double *eps_dev, double *res_dev, cudaStream_t st) {
    const rs_solver_cfg &c = S->cfg;
    const int n = c.nst;
    const size_t nn = (size_t)n * n;
    if (!S->psi64.p) {
        RS_TRY(S->psi64.alloc(sizeof(double) * (size_t)S->npts * n));
        RS_TRY(S->hpsi64.alloc(sizeof(double) * (size_t)S->npts * n));
        RS_TRY(S->rr64.alloc(sizeof(double) * (4 * nn + 16) + eigh_work_bytes(n)));
    }
    DevBuf cbuf;
    RS_TRY(cbuf.alloc(sizeof(double) * (2 * nn)));
    double *Sm = S->rr64.as<double>(), *h = Sm + nn, *Ui = h + nn, *T = Ui + nn;
    double *Y = cbuf.as<double>(), *C = Y + nn;
    int *status = reinterpret_cast<int *>(T + nn);
    void *ew = reinterpret_cast<void *>(T + nn + 16);
    double *P = S->psi64.as<double>(), *Q = S->hpsi64.as<double>();
    const int64_t total = S->npts * n;
    if (n_smooth > 0 && !(lam > 0)) {
        if (!(S->lam_max > 0)) RS_TRY(lambda_max_estimate(S, P, Q, st, &S->lam_max));
        lam = S->lam_max;
    }
    // FP64 orbitals (a widened copy of FP32 ones) and H applied in FP64
    if (c.dtype == RS_F32) {
        k_widen<<<1024, 256, 0, st>>>(S->psi.as<float>(), P, total);
        RS_LAUNCH_CHECK();
    } else {
        RS_CUDA(cudaMemcpyAsync(P, S->psi.p, sizeof(double) * (size_t)total, cudaMemcpyDeviceToDevice, st));
    }
    for (int b = 0; b < n; b += c.nb) RS_TRY(rs_ham_apply_block(S->h, P + b, n, Q + b, n, c.nb, RS_F64, st));
    if (n_smooth > 0) {
        // the step must damp every mode above the subspace: lam above the
        // largest current eigenvalue
        std::vector<double> e(n);
        RS_CUDA(cudaMemcpyAsync(e.data(), S->eig.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
        for (double v : e)
            if (!(lam > v)) return fail(RS_EINVAL, "rs_solver_certify_smoothed: lambda_max %g below an eigenvalue %g", lam, v);
    }
    for (int s = 0; s < n_smooth; ++s) {
        k_smooth_step<<<1024, 256, 0, st>>>(P, Q, S->eig.as<double>(), lam, n, total);
        RS_LAUNCH_CHECK();
        for (int b = 0; b < n; b += c.nb) RS_TRY(rs_ham_apply_block(S->h, P + b, n, Q + b, n, c.nb, RS_F64, st));
    }
    // h x = eps S x (Sec. VI, Eq. 7) with S = U^T U: the Ritz vectors are
    // Psi C with C = U^-1 Y, Y the eigenvectors of U^-T h U^-1
    RS_TRY(gram<double>(P, n, n, P, n, n, S->npts, S->dV, Sm, n, st));
    RS_TRY(gram<double>(P, n, n, Q, n, n, S->npts, S->dV, h, n, st));
    RS_TRY(symmetrize(Sm, n, n, st));
    RS_TRY(symmetrize(h, n, n, st));
    RS_TRY(cholesky(Sm, n, n, 1e-14, status, st));
    int bad = 0;
    RS_CUDA(cudaMemcpyAsync(&bad, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    if (bad) return fail(RS_ENOTSPD, "rs_solver_certify: the orbitals' overlap is not positive definite");
    RS_TRY(tri_inv(Sm, n, n, Ui, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, Ui, n, true, h, n, false, 0.0, T, n, st));
    RS_TRY(gemm_small(n, n, n, 1.0, T, n, false, Ui, n, false, 0.0, h, n, st));
    RS_TRY(symmetrize(h, n, n, st));
    RS_TRY(eigh(h, n, n, eps_dev, Y, n, 2, status, ew, st));
    RS_TRY(gemm_small(n, n, n, 1.0, Ui, n, false, Y, n, false, 0.0, C, n, st));
    // the Ritz vectors and H applied to them (rotated in place), their FP64
    // residual norms ||H x_k - eps_k x_k|| with <x_k|x_k> = 1
    RS_TRY(rowmul<double>(P, n, n, C, n, n, P, n, S->npts, 1.0, 0.0, st));
    RS_TRY(rowmul<double>(Q, n, n, C, n, n, Q, n, S->npts, 1.0, 0.0, st));
    RS_CUDA(cudaMemsetAsync(res_dev, 0, sizeof(double) * n, st));
    k_resid_norm2<<<dim3((unsigned)((n + 255) / 256), 512), 256, 0, st>>>(P, Q, n, n, eps_dev, S->npts, res_dev);
    k_sqrt_scale<<<(n + 255) / 256, 256, 0, st>>>(res_dev, n, S->dV);
    RS_LAUNCH_CHECK();
    // (the dense eigensolver's own sweep caps are not an error here: the FP64
    // residual norms measure the Ritz pairs whatever path produced them)
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

extern "C" int rs_solver_certify(rs_solver *S, double *eps_dev, double *res_dev, void *stream) {
    if (!S || !eps_dev || !res_dev) return fail(RS_EINVAL, "rs_solver_certify: null argument");
    return certify_impl(S, 0, 0.0, eps_dev, res_dev, (cudaStream_t)stream);
}

extern "C" int rs_solver_certify_smoothed(rs_solver *S, int n_smooth, double lambda_max, double *eps_dev,
                                          double *res_dev, void *stream) {
    if (!S || !eps_dev || !res_dev) return fail(RS_EINVAL, "rs_solver_certify_smoothed: null argument");
    if (n_smooth < 0 || n_smooth > 16) return fail(RS_EINVAL, "rs_solver_certify_smoothed: n_smooth must be in 0 .. 16");
    if (!std::isfinite(lambda_max)) return fail(RS_EINVAL, "rs_solver_certify_smoothed: lambda_max must be finite");
    return certify_impl(S, n_smooth, lambda_max, eps_dev, res_dev, (cudaStream_t)stream);
}

extern "C" int rs_solver_rayleigh_ritz_f64(rs_solver *S, double *eps_dev, void *stream) {
    if (!S || !eps_dev) return fail(RS_EINVAL, "rs_solver_rayleigh_ritz_f64: null argument");
    return rayleigh_ritz_f64_impl(S, eps_dev, (cudaStream_t)stream);
}

extern "C" int rs_solver_create(rs_ham *h, const rs_solver_cfg *cfg, const void *Psi0_dev, void *stream,
                                rs_solver **out) {
    if (!h || !cfg || !Psi0_dev || !out) return fail(RS_EINVAL, "rs_solver_create: null argument");
    const rs_solver_cfg c = *cfg;
    if (c.nb < 1 || c.nb > 64 || (c.nb & (c.nb - 1))) return fail(RS_EINVAL, "rs_solver_create: nb must be a power of two <= 64");
    if (c.nst < c.nb || c.nst % c.nb) return fail(RS_EINVAL, "rs_solver_create: nst must be a multiple of nb");
    if (c.dtype != RS_F64 && c.dtype != RS_F32) return fail(RS_EINVAL, "rs_solver_create: bad dtype");
    if (c.precond < RS_PRECOND_NONE || c.precond > RS_PRECOND_LEARNED) return fail(RS_EINVAL, "rs_solver_create: bad precond");
    if (!(c.tol > 0)) return fail(RS_EINVAL, "rs_solver_create: tol must be > 0");
    if (c.n_wanted < 0 || c.n_wanted > c.nst) return fail(RS_EINVAL, "rs_solver_create: n_wanted must be in 0 .. nst");
    if (c.stall_sweeps < 0 || (c.stall_sweeps > 0 && !(c.stall_ratio > 0 && c.stall_ratio <= 1)))
        return fail(RS_EINVAL, "rs_solver_create: stall_sweeps must be >= 0 and stall_ratio in (0, 1]");
    if (c.rr64_every < 0 || !(c.rr64_below >= 0) || !(c.rr64_always >= 0))
        return fail(RS_EINVAL, "rs_solver_create: bad FP64 Rayleigh-Ritz schedule");
    if (c.method != RS_EIG_BLOCK_CG && c.method != RS_EIG_RMMDIIS) return fail(RS_EINVAL, "rs_solver_create: bad method");
    if (c.rmm_steps < 0 || c.rmm_steps > RMM_MAXK - 1)
        return fail(RS_EINVAL, "rs_solver_create: rmm_steps must be in 0 .. %d", RMM_MAXK - 1);
    *out = nullptr;
    rs_solver *S = new (std::nothrow) rs_solver;
    if (!S) return fail(RS_ENOMEM, "host allocation failed");
    auto bail = [&](int rc) {
        delete S;
        return rc;
    };
    S->h = h;
    S->cfg = c;
    S->npts = ham_npts(h);
    S->dV = ham_dV(h);
    S->es = c.dtype == RS_F64 ? 8 : 4;
    S->nblk = c.nst / c.nb;
    S->has_p.assign(S->nblk, 0);
    const size_t big = (size_t)S->npts * c.nst * S->es, zb = (size_t)S->npts * 3 * c.nb * S->es;
    const bool rmm = c.method == RS_EIG_RMMDIIS;
    S->rmm_M = c.rmm_steps > 0 ? c.rmm_steps : 3;
    int rc;
    if ((rc = S->psi.alloc(big)) || (rc = S->hpsi.alloc(big)) ||
        (rc = S->la.alloc(LaWork::bytes(c.nst))) || (rc = S->eig.alloc(sizeof(double) * c.nst)) ||
        (rc = S->res.alloc(sizeof(double) * c.nst)))
        return bail(rc);
    if (!rmm && ((rc = S->P.alloc(big)) || (rc = S->Z.alloc(zb)) || (rc = S->HZ.alloc(zb)) ||
                 (rc = S->R.alloc((size_t)S->npts * c.nb * S->es))))
        return bail(rc);
    if (rmm && ((rc = S->rmm_hist.alloc((size_t)(3 * (S->rmm_M + 1) + 5) * S->npts * c.nb * S->es)) ||
                (rc = S->rmm_small.alloc(sizeof(double) * 64 * (MD_MAX + 2 * RMM_MAXK * RMM_MAXK + RMM_MAXK + 2)))))
        return bail(rc);
    if (c.dtype == RS_F32) {
        const int64_t need = std::max({umma_work_bytes(c.nst, 2 * c.nb, S->npts), umma_work_bytes(S->npts, c.nst, c.nst),
                                       umma_work_bytes(3 * c.nb, 3 * c.nb, S->npts),
                                       umma_work_bytes(c.nst, c.nst, S->npts)});
        if ((rc = S->tcbuf.alloc((size_t)need + 256))) return bail(rc);
        // the Gram-Schmidt splits of Psi, one per contraction layout
        if ((rc = S->gs_tbuf.alloc((size_t)umma_split_cache_bytes(true, S->npts, c.nst)))) return bail(rc);
        if ((rc = S->gs_nbuf.alloc((size_t)umma_split_cache_bytes(false, S->npts, c.nst)))) return bail(rc);
        S->gs_t.buf = S->gs_tbuf.p;
        S->gs_n.buf = S->gs_nbuf.p;
        S->tc.p = S->tcbuf.p;
        S->tc.bytes = need;
        S->tc.err = reinterpret_cast<int *>((char *)S->tcbuf.p + need);
        S->tc.inner = true;
        if (cudaMemset(S->tc.err, 0, sizeof(int)) != cudaSuccess) return bail(fail(RS_ECUDA, "cudaMemset failed"));
    }
    const int n3 = 3 * c.nb;
    const size_t smallbytes = sizeof(double) * (512 + (size_t)c.nst * 2 * c.nb + 7 * (size_t)n3 * n3 + n3 + (size_t)n3 * c.nb) +
                              64 + eigh_work_bytes(n3);
    if ((rc = S->small.alloc(smallbytes))) return bail(rc);
    double *d = S->small.as<double>();
    S->dots = d;
    S->M = d + 512;
    S->G = S->M + (size_t)c.nst * 2 * c.nb;
    S->A = S->G + (size_t)n3 * n3;
    S->U = S->A + (size_t)n3 * n3;
    S->Ui = S->U + (size_t)n3 * n3;
    S->T1 = S->Ui + (size_t)n3 * n3;
    S->At = S->T1 + (size_t)n3 * n3;
    S->Yv = S->At + (size_t)n3 * n3;
    S->mu = S->Yv + (size_t)n3 * n3;
    S->C = S->mu + n3;
    S->status = reinterpret_cast<int *>(S->C + (size_t)n3 * c.nb);
    S->eighw = reinterpret_cast<void *>(S->C + (size_t)n3 * c.nb + 8);
    S->pc = Precond::create(c.precond, c.filter_alpha, S->npts, c.nb, c.dtype);
    if (!S->pc) return bail(fail(RS_EINVAL, "rs_solver_create: preconditioner %d unavailable", c.precond));
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(S->psi.p, Psi0_dev, big, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        (S->P.p && cudaMemsetAsync(S->P.p, 0, big, st) != cudaSuccess) ||
        cudaMemsetAsync(S->res.p, 0, sizeof(double) * c.nst, st) != cudaSuccess)
        return bail(fail(RS_ECUDA, "rs_solver_create: copy failed"));
    if ((rc = orthonormalize_impl(S->npts, S->dV, S->psi.p, c.nst, c.nst, c.dtype, S->la.p, st, S->tc))) return bail(rc);
    if ((rc = subspace_diag_impl(h, S->psi.p, S->hpsi.p, c.nst, c.nst, c.dtype, c.nb, S->la.p, S->eig.as<double>(), st,
                                 S->tc)))
        return bail(rc);
    if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(RS_ECUDA, "rs_solver_create: sync failed"));
    *out = S;
    return RS_OK;
}

extern "C" int rs_eigensolver_step(rs_solver *S, double *eps_dev, double *resnorm_dev, int *n_converged, void *stream) {
    if (!S) return fail(RS_EINVAL, "rs_eigensolver_step: null solver");
    cudaStream_t st = (cudaStream_t)stream;
    const rs_solver_cfg &c = S->cfg;
    const bool rmm = c.method == RS_EIG_RMMDIIS;
    for (int b = 0; b < S->nblk; ++b) RS_TRY(rmm ? rmm_block_step(S, b, st) : block_step(S, b, st));
    RS_TRY(orthonormalize_impl(S->npts, S->dV, S->psi.p, c.nst, c.nst, c.dtype, S->la.p, st, S->tc));
    LaWork w(S->la.p, c.nst);
    if (!rmm) RS_TRY(rotate_inplace(S->P.p, c.nst, c.nst, w.Ui, S->npts, c.dtype, st, S->tc));
    RS_TRY(subspace_diag_impl(S->h, S->psi.p, S->hpsi.p, c.nst, c.nst, c.dtype, c.nb, S->la.p, S->eig.as<double>(), st,
                              S->tc));
    if (!rmm) RS_TRY(rotate_inplace(S->P.p, c.nst, c.nst, w.xi, S->npts, c.dtype, st, S->tc));
    if (eps_dev) RS_CUDA(cudaMemcpyAsync(eps_dev, S->eig.p, sizeof(double) * c.nst, cudaMemcpyDeviceToDevice, st));
    if (resnorm_dev) RS_CUDA(cudaMemcpyAsync(resnorm_dev, S->res.p, sizeof(double) * c.nst, cudaMemcpyDeviceToDevice, st));
    std::vector<double> res(c.nst);
    RS_CUDA(cudaMemcpyAsync(res.data(), S->res.p, sizeof(double) * c.nst, cudaMemcpyDeviceToHost, st));
    // status words of the bounded device waits: the tensor-core pipeline and
    // the H psi ring (a wait that gave up leaves that launch's result incomplete)
    int tcerr = 0, ringerr = 0;
    if (S->tc.err) RS_CUDA(cudaMemcpyAsync(&tcerr, S->tc.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (int *rw = ham_status_word(S->h)) RS_CUDA(cudaMemcpyAsync(&ringerr, rw, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    if (tcerr) return fail(RS_ETIMEOUT, "eigensolver: a tensor-core pipeline wait timed out");
    if (ringerr) return fail(RS_ETIMEOUT, "eigensolver: an H psi pipeline wait timed out");
    ++S->sweeps;
    const int nw = c.n_wanted > 0 ? c.n_wanted : c.nst;
    double rmax = 0;
    for (int k = 0; k < nw; ++k) rmax = std::max(rmax, res[k]);
    S->max_res = rmax;
    if (n_converged) {
        int k = 0;
        for (double r : res) k += r <= c.tol;
        *n_converged = k;
    }
    // the learned preconditioner gives way to the plain filter once it stops
    // reducing the largest wanted residual (stall_sweeps sweeps in a row
    // without a drop below stall_ratio times the best so far)
    if (S->pc->kind() == RS_PRECOND_LEARNED && c.stall_sweeps > 0 && !S->fallback_sweep) {
        if (rmax < c.stall_ratio * S->best) {
            S->best = rmax;
            S->stall = 0;
        } else if (++S->stall >= c.stall_sweeps) {
            Precond *p = Precond::create(RS_PRECOND_FILTER, c.filter_alpha, S->npts, c.nb, c.dtype);
            if (!p) return fail(RS_ENOMEM, "eigensolver: filter fallback unavailable");
            delete S->pc;   // the sweep above is complete (the stream was synchronised)
            S->pc = p;
            S->fallback_sweep = S->sweeps;
        }
    }
    // FP32 solvers: eigenvalues from the closing FP64 Rayleigh-Ritz, taken at
    // every sweep once the largest wanted residual is <= rr64_always and every
    // rr64_every sweeps once it is <= rr64_below
    S->eps_f64 = c.dtype == RS_F64;
    if (c.dtype == RS_F32 && c.rr64_every > 0 &&
        (rmax <= c.rr64_always || (rmax <= c.rr64_below && S->sweeps % c.rr64_every == 0))) {
        double *out = eps_dev;
        if (!out) {
            if (!S->eps64.p) RS_TRY(S->eps64.alloc(sizeof(double) * c.nst));
            out = S->eps64.as<double>();
        }
        RS_TRY(rayleigh_ritz_f64_impl(S, out, st));
        S->eps_f64 = 1;
    }
    return RS_OK;
}

extern "C" int rs_solver_stats(rs_solver *S, rs_solver_stats_t *out) {
    if (!S || !out) return fail(RS_EINVAL, "rs_solver_stats: null argument");
    out->sweeps = S->sweeps;
    out->eps_f64 = S->eps_f64;
    out->precond = S->pc->kind();
    out->fallback_sweep = S->fallback_sweep;
    out->max_residual = S->max_res;
    out->train_target_seconds = S->train_target_s;
    out->train_fit_seconds = S->train_fit_s;
    out->lambda_max = S->lam_max;
    return RS_OK;
}

template <typename T>
__global__ void k_ritz_residual(const T *__restrict__ X, const T *__restrict__ HX, int64_t ld, const double *__restrict__ eps,
                                int first, int ncols, int64_t npts, T *__restrict__ R, int64_t ldr) {
    const int rows = blockDim.x / ncols, k = threadIdx.x % ncols, r = threadIdx.x / ncols;
    if (r >= rows) return;
    const T e = (T)eps[first + k];
    for (int64_t p = blockIdx.x * (int64_t)rows + r; p < npts; p += (int64_t)gridDim.x * rows)
        R[p * ldr + k] = HX[p * ld + first + k] - e * X[p * ld + first + k];
}

extern "C" int rs_solver_residual(rs_solver *S, int first, int ncols, void *R_dev, int64_t ldr, void *stream) {
    if (!S || !R_dev) return fail(RS_EINVAL, "rs_solver_residual: null argument");
    if (first < 0 || ncols < 1 || first + ncols > S->cfg.nst || ldr < ncols)
        return fail(RS_EINVAL, "rs_solver_residual: bad state range");
    if (ncols > 256) return fail(RS_EINVAL, "rs_solver_residual: at most 256 columns per call");
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = elem_blocks(S->npts, ncols);
    if (S->cfg.dtype == RS_F64)
        k_ritz_residual<double><<<blocks, 256, 0, st>>>(S->psi.as<double>(), S->hpsi.as<double>(), S->cfg.nst,
                                                        S->eig.as<double>(), first, ncols, S->npts, (double *)R_dev, ldr);
    else
        k_ritz_residual<float><<<blocks, 256, 0, st>>>(S->psi.as<float>(), S->hpsi.as<float>(), S->cfg.nst,
                                                       S->eig.as<double>(), first, ncols, S->npts, (float *)R_dev, ldr);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

extern "C" int rs_solver_psi(rs_solver *S, void **psi_dev) {
    if (!S || !psi_dev) return fail(RS_EINVAL, "rs_solver_psi: null argument");
    *psi_dev = S->psi.p;
    return RS_OK;
}

// Keeps a copy of the learned weights in the solver (saved by
// rs_precond_save, reinstated when the learned preconditioner is selected
// again) and hands them to the current preconditioner when it is the learned one.
static int store_weights(rs_solver *S, const float *w_dev, cudaStream_t st) {
    if (!S->wlearn.p) RS_TRY(S->wlearn.alloc(sizeof(float) * LEARNED_WEIGHTS));
    if (w_dev != S->wlearn.as<float>())
        RS_CUDA(cudaMemcpyAsync(S->wlearn.p, w_dev, sizeof(float) * LEARNED_WEIGHTS, cudaMemcpyDeviceToDevice, st));
    S->has_wlearn = true;
    if (S->pc->kind() == RS_PRECOND_LEARNED) RS_TRY(S->pc->set_weights(S->wlearn.as<float>(), st));
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

extern "C" int rs_solver_set_precond_weights(rs_solver *S, const float *w_dev) {
    if (!S || !w_dev) return fail(RS_EINVAL, "rs_solver_set_precond_weights: null argument");
    if (S->pc->kind() != RS_PRECOND_LEARNED)
        return fail(RS_EINVAL, "rs_solver_set_precond_weights: the solver's preconditioner is not the learned one");
    RS_CUDA(cudaDeviceSynchronize());   // the caller's weights are written on any stream
    return store_weights(S, w_dev, nullptr);
}

extern "C" int rs_precond_train(rs_solver *S, const rs_grid *g, const rs_learn_cfg *cfg, const float *w_init_dev,
                                float *loss_host, void *stream) {
    if (!S || !g || !cfg) return fail(RS_EINVAL, "rs_precond_train: null argument");
    const rs_learn_cfg c = *cfg;
    const rs_solver_cfg &sc = S->cfg;
    if (sc.dtype != RS_F32) return fail(RS_EINVAL, "rs_precond_train: the learned preconditioner needs an RS_F32 solver");
    if (S->pc->kind() != RS_PRECOND_LEARNED) return fail(RS_EINVAL, "rs_precond_train: the solver's preconditioner is not the learned one");
    if (g->npts != S->npts) return fail(RS_EINVAL, "rs_precond_train: grid of another size");
    if (c.n_res < 1 || c.n_res > sc.nst || c.n_res > 256 || c.cg_iters < 0 || c.cg_iters > 10000 || !(c.sigma > 0) ||
        c.train.n_tiles < 1 || c.train.batch < 1 || c.train.epochs < 0 || c.train.tile < 1 || c.train.tile > 58 ||
        !(c.train.lr > 0))
        return fail(RS_EINVAL, "rs_precond_train: bad configuration");
    if (!w_init_dev && !S->has_wlearn) return fail(RS_EINVAL, "rs_precond_train: no initial weights");
    cudaStream_t st = (cudaStream_t)stream;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    // the residual columns, padded to the CG block width (a power of two <= 64)
    int w = 1;
    while (w < std::min(c.n_res, 64)) w <<= 1;
    const int chunks = (c.n_res + w - 1) / w, ld = chunks * w;
    const int64_t np = S->npts;
    DevBuf R, X, work, nrm;
    RS_TRY(R.alloc(sizeof(float) * (size_t)np * ld));
    RS_TRY(X.alloc(sizeof(float) * (size_t)np * ld));
    RS_TRY(work.alloc((size_t)rs_cg_workspace_bytes(np, w, RS_F32)));
    RS_TRY(nrm.alloc(sizeof(double) * 256));
    const int ncols = std::min(ld, sc.nst);
    RS_TRY(rs_solver_residual(S, 0, ncols, R.p, ld, st));
    if (ncols < ld)
        RS_CUDA(cudaMemset2DAsync(R.as<float>() + ncols, sizeof(float) * ld, 0, sizeof(float) * (ld - ncols), (size_t)np, st));
    // targets: cg_iters conjugate-gradient iterations on (-1/2 Lap + sigma) X = R,
    // the operator applied by a Hamiltonian on the same grid with V = sigma
    {
        std::vector<double> Vs((size_t)np, c.sigma);
        rs_ham *hs = nullptr;
        RS_TRY(rs_ham_create(g, Vs.data(), nullptr, 4, &hs));
        int rc = RS_OK;
        for (int k = 0; k < chunks && rc == RS_OK; ++k)
            rc = rs_shifted_poisson_cg(hs, R.as<float>() + k * w, X.as<float>() + k * w, ld, w, c.cg_iters, RS_F32, work.p, st);
        if (rc == RS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(RS_ECUDA, "rs_precond_train: CG failed");
        rs_ham_destroy(hs);
        RS_TRY(rc);
    }
    // the eigensolver uses only the direction of K r: every target column is
    // scaled to unit rms, like the network's input r / rms(r); unscaled
    // targets (about 1/50 of the input) would let an output near zero that
    // carries no direction minimise the loss
    RS_TRY(coldots(RS_F32, X.p, ld, X.p, ld, c.n_res, np, nrm.as<double>(), st));
    k_scale_cols<float><<<elem_blocks(np, c.n_res), 256, 0, st>>>(X.as<float>(), ld, c.n_res, np, nrm.as<double>(),
                                                                  1.0 / (double)np);
    RS_LAUNCH_CHECK();
    RS_CUDA(cudaStreamSynchronize(st));
    const auto t1 = clk::now();
    DevBuf wt;
    RS_TRY(wt.alloc(sizeof(float) * LEARNED_WEIGHTS));
    RS_CUDA(cudaMemcpyAsync(wt.p, w_init_dev ? w_init_dev : S->wlearn.as<float>(), sizeof(float) * LEARNED_WEIGHTS,
                            cudaMemcpyDeviceToDevice, st));
    RS_TRY(train_pairs_impl(S->h, g, R.as<float>(), X.as<float>(), ld, c.n_res, c.train, wt.as<float>(), loss_host, st));
    RS_TRY(store_weights(S, wt.as<float>(), st));
    S->train_target_s = std::chrono::duration<double>(t1 - t0).count();
    S->train_fit_s = std::chrono::duration<double>(clk::now() - t1).count();
    return RS_OK;
}

// Weight file: the 4 bytes "RSNN", then little-endian uint32 version (1),
// uint32 count (2160), count FP32 values, and the uint32 FNV-1a hash of the
// value bytes.
static uint32_t fnv1a(const unsigned char *p, size_t n) {
    uint32_t h = 2166136261u;
    for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 16777619u;
    return h;
}
static void put_u32(unsigned char *d, uint32_t v) {
    for (int i = 0; i < 4; ++i) d[i] = (unsigned char)(v >> (8 * i));
}
static uint32_t get_u32(const unsigned char *d) {
    return (uint32_t)d[0] | (uint32_t)d[1] << 8 | (uint32_t)d[2] << 16 | (uint32_t)d[3] << 24;
}

extern "C" int rs_precond_save(rs_solver *S, const char *path) {
    if (!S || !path) return fail(RS_EINVAL, "rs_precond_save: null argument");
    if (!S->has_wlearn) return fail(RS_EINVAL, "rs_precond_save: no learned weights set or trained");
    std::vector<float> w(LEARNED_WEIGHTS);
    RS_CUDA(cudaMemcpy(w.data(), S->wlearn.p, sizeof(float) * LEARNED_WEIGHTS, cudaMemcpyDeviceToHost));
    const size_t nv = sizeof(float) * LEARNED_WEIGHTS;
    std::vector<unsigned char> buf(12 + nv + 4);
    memcpy(buf.data(), "RSNN", 4);
    put_u32(buf.data() + 4, 1);
    put_u32(buf.data() + 8, LEARNED_WEIGHTS);
    for (int i = 0; i < LEARNED_WEIGHTS; ++i) {
        uint32_t u;
        memcpy(&u, &w[i], 4);
        put_u32(buf.data() + 12 + 4 * i, u);
    }
    put_u32(buf.data() + 12 + nv, fnv1a(buf.data() + 12, nv));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(RS_EINVAL, "rs_precond_save: cannot open %s", path);
    const bool ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    if (fclose(f) != 0 || !ok) return fail(RS_EINVAL, "rs_precond_save: write to %s failed", path);
    return RS_OK;
}

extern "C" int rs_precond_load(rs_solver *S, const char *path) {
    if (!S || !path) return fail(RS_EINVAL, "rs_precond_load: null argument");
    if (S->pc->kind() != RS_PRECOND_LEARNED)
        return fail(RS_EINVAL, "rs_precond_load: the solver's preconditioner is not the learned one");
    const size_t nv = sizeof(float) * LEARNED_WEIGHTS;
    std::vector<unsigned char> buf(12 + nv + 4 + 1);
    FILE *f = fopen(path, "rb");
    if (!f) return fail(RS_EINVAL, "rs_precond_load: cannot open %s", path);
    const size_t got = fread(buf.data(), 1, buf.size(), f);
    fclose(f);
    if (got != 12 + nv + 4 || memcmp(buf.data(), "RSNN", 4) != 0 || get_u32(buf.data() + 4) != 1 ||
        get_u32(buf.data() + 8) != (uint32_t)LEARNED_WEIGHTS)
        return fail(RS_EINVAL, "rs_precond_load: %s is not a weight file of this library", path);
    if (get_u32(buf.data() + 12 + nv) != fnv1a(buf.data() + 12, nv))
        return fail(RS_EINVAL, "rs_precond_load: checksum mismatch in %s", path);
    std::vector<float> w(LEARNED_WEIGHTS);
    for (int i = 0; i < LEARNED_WEIGHTS; ++i) {
        const uint32_t u = get_u32(buf.data() + 12 + 4 * i);
        memcpy(&w[i], &u, 4);
        if (!std::isfinite(w[i])) return fail(RS_ENAN, "rs_precond_load: non-finite weight in %s", path);
    }
    RS_CUDA(cudaDeviceSynchronize());   // no queued sweep still reads the weights
    if (!S->wlearn.p) RS_TRY(S->wlearn.alloc(sizeof(float) * LEARNED_WEIGHTS));
    RS_CUDA(cudaMemcpy(S->wlearn.p, w.data(), nv, cudaMemcpyHostToDevice));
    return store_weights(S, S->wlearn.as<float>(), nullptr);
}

extern "C" int rs_solver_set_precond(rs_solver *S, int precond) {
    if (!S) return fail(RS_EINVAL, "rs_solver_set_precond: null solver");
    if (precond < RS_PRECOND_NONE || precond > RS_PRECOND_LEARNED)
        return fail(RS_EINVAL, "rs_solver_set_precond: bad preconditioner");
    Precond *p = Precond::create(precond, S->cfg.filter_alpha, S->npts, S->cfg.nb, S->cfg.dtype);
    if (!p) return fail(RS_EINVAL, "rs_solver_set_precond: preconditioner %d unavailable", precond);
    RS_CUDA(cudaDeviceSynchronize());   // no sweep still uses the old one
    delete S->pc;
    S->pc = p;
    S->cfg.precond = precond;
    // a learned preconditioner selected again takes the weights last set
    if (precond == RS_PRECOND_LEARNED && S->has_wlearn) RS_TRY(store_weights(S, S->wlearn.as<float>(), nullptr));
    return RS_OK;
}

extern "C" int rs_solver_set_precond_cg(rs_solver *S, rs_ham *shifted, int n_iter) {
    if (!S || !shifted) return fail(RS_EINVAL, "rs_solver_set_precond_cg: null argument");
    if (n_iter < 1 || n_iter > 200) return fail(RS_EINVAL, "rs_solver_set_precond_cg: n_iter must be in 1 .. 200");
    if (ham_npts(shifted) != S->npts) return fail(RS_EINVAL, "rs_solver_set_precond_cg: grid size differs");
    Precond *p = Precond::create_cg(shifted, n_iter, S->npts, S->cfg.nb, S->cfg.dtype);
    if (!p) return fail(RS_ENOMEM, "rs_solver_set_precond_cg: allocation failed");
    RS_CUDA(cudaDeviceSynchronize());   // no sweep still uses the old one
    delete S->pc;
    S->pc = p;
    return RS_OK;
}

// Checkpoint file: "RSCK", then little-endian uint32 version (1), int64
// npts, int32 nst, nb, dtype, method, sweeps, uint32 has-P flag, the
// orbitals, H applied to them and (block CG) the search directions as raw
// arrays [npts][nst] of the solver's element type, the eigenvalues and the
// residual norms (double [nst] each), one byte per block (search direction
// present), and the uint32 FNV-1a hash of everything after the magic.
namespace {
struct CkWriter {
    FILE *f;
    uint32_t h = 2166136261u;
    bool ok = true;
    void put(const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 16777619u;
        ok = ok && fwrite(p, 1, n, f) == n;
    }
};
struct CkReader {
    FILE *f;
    uint32_t h = 2166136261u;
    bool ok = true;
    void get(void *p, size_t n) {
        ok = ok && fread(p, 1, n, f) == n;
        const unsigned char *c = (const unsigned char *)p;
        for (size_t i = 0; ok && i < n; ++i) h = (h ^ c[i]) * 16777619u;
    }
};
}  // namespace

extern "C" int rs_solver_checkpoint_save(rs_solver *S, const char *path) {
    if (!S || !path) return fail(RS_EINVAL, "rs_solver_checkpoint_save: null argument");
    const rs_solver_cfg &c = S->cfg;
    const size_t big = (size_t)S->npts * c.nst * S->es;
    std::vector<unsigned char> host(big);
    FILE *f = fopen(path, "wb");
    if (!f) return fail(RS_EINVAL, "rs_solver_checkpoint_save: cannot open %s", path);
    CkWriter w{f};
    if (fwrite("RSCK", 1, 4, f) != 4) w.ok = false;
    const uint32_t ver = 1, hp = S->P.p ? 1u : 0u;
    const int64_t np = S->npts;
    const int32_t hdr[5] = {c.nst, c.nb, c.dtype, c.method, S->sweeps};
    w.put(&ver, 4);
    w.put(&np, 8);
    w.put(hdr, sizeof(hdr));
    w.put(&hp, 4);
    int rc = RS_OK;
    for (DevBuf *b : {&S->psi, &S->hpsi, &S->P}) {
        if (b == &S->P && !hp) continue;
        if (cudaMemcpy(host.data(), b->p, big, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = fail(RS_ECUDA, "rs_solver_checkpoint_save: copy failed");
            break;
        }
        w.put(host.data(), big);
    }
    std::vector<double> e(c.nst), r(c.nst);
    if (rc == RS_OK && (cudaMemcpy(e.data(), S->eig.p, 8 * c.nst, cudaMemcpyDeviceToHost) != cudaSuccess ||
                        cudaMemcpy(r.data(), S->res.p, 8 * c.nst, cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = fail(RS_ECUDA, "rs_solver_checkpoint_save: copy failed");
    if (rc == RS_OK) {
        w.put(e.data(), 8 * e.size());
        w.put(r.data(), 8 * r.size());
        w.put(S->has_p.data(), S->has_p.size());
        const uint32_t hh = w.h;
        w.ok = w.ok && fwrite(&hh, 1, 4, f) == 4;
    }
    if (fclose(f) != 0) w.ok = false;
    if (rc != RS_OK) return rc;
    if (!w.ok) return fail(RS_EINVAL, "rs_solver_checkpoint_save: write to %s failed", path);
    return RS_OK;
}

extern "C" int rs_solver_checkpoint_load(rs_solver *S, const char *path) {
    if (!S || !path) return fail(RS_EINVAL, "rs_solver_checkpoint_load: null argument");
    const rs_solver_cfg &c = S->cfg;
    const size_t big = (size_t)S->npts * c.nst * S->es;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(RS_EINVAL, "rs_solver_checkpoint_load: cannot open %s", path);
    char magic[4] = {0, 0, 0, 0};
    CkReader r{f};
    r.ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, "RSCK", 4) == 0;
    uint32_t ver = 0, hp = 0;
    int64_t np = 0;
    int32_t hdr[5] = {0, 0, 0, 0, 0};
    r.get(&ver, 4);
    r.get(&np, 8);
    r.get(hdr, sizeof(hdr));
    r.get(&hp, 4);
    const bool match = r.ok && ver == 1 && np == S->npts && hdr[0] == c.nst && hdr[1] == c.nb && hdr[2] == c.dtype &&
                       hdr[3] == c.method && hp == (S->P.p ? 1u : 0u);
    if (!match) {
        fclose(f);
        return fail(RS_EINVAL, "rs_solver_checkpoint_load: %s is not a checkpoint of a solver of this shape", path);
    }
    std::vector<unsigned char> psi(big), hpsi(big), P(hp ? big : 0);
    std::vector<double> e(c.nst), res(c.nst);
    std::vector<char> has_p(S->has_p.size());
    r.get(psi.data(), big);
    r.get(hpsi.data(), big);
    if (hp) r.get(P.data(), big);
    r.get(e.data(), 8 * e.size());
    r.get(res.data(), 8 * res.size());
    r.get(has_p.data(), has_p.size());
    uint32_t stored = 0;
    const uint32_t h = r.h;
    const bool tail = fread(&stored, 1, 4, f) == 4;
    fclose(f);
    if (!r.ok || !tail || stored != h) return fail(RS_EINVAL, "rs_solver_checkpoint_load: %s is damaged", path);
    RS_CUDA(cudaDeviceSynchronize());
    RS_CUDA(cudaMemcpy(S->psi.p, psi.data(), big, cudaMemcpyHostToDevice));
    RS_CUDA(cudaMemcpy(S->hpsi.p, hpsi.data(), big, cudaMemcpyHostToDevice));
    if (hp) RS_CUDA(cudaMemcpy(S->P.p, P.data(), big, cudaMemcpyHostToDevice));
    RS_CUDA(cudaMemcpy(S->eig.p, e.data(), 8 * e.size(), cudaMemcpyHostToDevice));
    RS_CUDA(cudaMemcpy(S->res.p, res.data(), 8 * res.size(), cudaMemcpyHostToDevice));
    S->has_p = has_p;
    S->sweeps = hdr[4];
    return RS_OK;
}

extern "C" int rs_solver_set_potential(rs_solver *S, const double *V_dev, void *stream) {
    if (!S || !V_dev) return fail(RS_EINVAL, "rs_solver_set_potential: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const rs_solver_cfg &c = S->cfg;
    RS_TRY(rs_ham_set_potential(S->h, V_dev, st));
    // the current subspace rediagonalised with the new H; search directions dropped
    RS_TRY(subspace_diag_impl(S->h, S->psi.p, S->hpsi.p, c.nst, c.nst, c.dtype, c.nb, S->la.p, S->eig.as<double>(), st,
                              S->tc));
    if (S->P.p) RS_CUDA(cudaMemsetAsync(S->P.p, 0, S->P.bytes, st));
    std::fill(S->has_p.begin(), S->has_p.end(), 0);
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

namespace rs {
void solver_view(rs_solver *S, SolverView *v) {
    v->psi = S->psi.p;
    v->eig = S->eig.as<double>();
    v->nst = S->cfg.nst;
    v->dtype = S->cfg.dtype;
    v->npts = S->npts;
    v->dV = S->dV;
}
}  // namespace rs

extern "C" int rs_solver_destroy(rs_solver *S) {
    delete S;
    return RS_OK;
}

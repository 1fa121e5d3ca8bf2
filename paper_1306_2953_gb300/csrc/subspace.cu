// C-ABI entry points of Sec. VI: overlap (Eq. 5), Cholesky orthogonalisation
// (Eq. 6) and subspace diagonalisation (Eqs. 7-8).  Everything stays on the
// device; the only host interaction is reading a status word at the end of
// the blocking calls.
#include <algorithm>
#include <cmath>

#include "device.h"
#include "ham.h"
#include "linalg.h"
#include "umma.h"

using namespace rs;

namespace {

template <typename T> int overlap_t(const void *X, int64_t ldx, int nx, const void *Y, int64_t ldy, int ny,
                                    int64_t npts, double dV, double *S, int64_t lds, cudaStream_t st) {
    return gram<T>((const T *)X, ldx, nx, (const T *)Y, ldy, ny, npts, dV, S, lds, st);
}

int check_block(const void *p, int64_t ld, int n, int dtype) {
    if (!p) return fail(RS_EINVAL, "null device pointer");
    if (n < 1 || ld < n) return fail(RS_EINVAL, "bad column count or leading dimension");
    if (dtype != RS_F64 && dtype != RS_F32) return fail(RS_EINVAL, "bad dtype");
    return RS_OK;
}

}  // namespace

extern "C" int rs_overlap_block(const rs_grid *g, const void *X_dev, int64_t ldx, int nx, const void *Y_dev,
                                int64_t ldy, int ny, double *S_dev, int64_t lds, int dtype, void *stream) {
    if (!g || !S_dev) return fail(RS_EINVAL, "rs_overlap_block: null argument");
    RS_TRY(check_block(X_dev, ldx, nx, dtype));
    RS_TRY(check_block(Y_dev, ldy, ny, dtype));
    if (lds < ny) return fail(RS_EINVAL, "rs_overlap_block: lds < ny");
    const double dV = g->h * g->h * g->h;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == RS_F64) return overlap_t<double>(X_dev, ldx, nx, Y_dev, ldy, ny, g->npts, dV, S_dev, lds, st);
    return overlap_t<float>(X_dev, ldx, nx, Y_dev, ldy, ny, g->npts, dV, S_dev, lds, st);
}

extern "C" int64_t rs_linalg_workspace_bytes(int nst) {
    if (nst < 1) return -1;
    return (int64_t)LaWork::bytes(nst);
}

namespace rs {

namespace {
bool tc_grams(const TcWork &tc, int n, int64_t npts) {
    return tc.inner && tc.p && tc.bytes >= umma_work_bytes(n, n, npts);
}
}  // namespace

int rotate_inplace(void *Psi, int64_t ld, int n, const double *C, int64_t npts, int dtype, cudaStream_t st,
                   const TcWork &tc) {
    if (dtype == RS_F64) return rowmul<double>((const double *)Psi, ld, n, C, n, n, (double *)Psi, ld, npts, 1.0, 0.0, st);
    if (tc.p && tc.bytes >= umma_work_bytes(npts, n, n))
        return umma_rowmul((const float *)Psi, ld, n, C, n, n, (float *)Psi, ld, npts, 1.0, 0.0, tc.p, tc.err, st);
    return rowmul<float>((const float *)Psi, ld, n, C, n, n, (float *)Psi, ld, npts, 1.0, 0.0, st);
}

// Orthonormalise Psi in place; Ui (n x n) receives U^-1.  Blocking.
int orthonormalize_impl(int64_t npts, double dV, void *Psi, int64_t ld, int n, int dtype, void *work, cudaStream_t st,
                        const TcWork &tc) {
    LaWork w(work, n);
    if (dtype == RS_F64)
        RS_TRY(gram<double>((const double *)Psi, ld, n, (const double *)Psi, ld, n, npts, dV, w.U, n, st));
    else if (tc_grams(tc, n, npts))
        RS_TRY(umma_gram((const float *)Psi, ld, n, (const float *)Psi, ld, n, npts, dV, w.U, n, tc.p, tc.err, st));
    else
        RS_TRY(gram<float>((const float *)Psi, ld, n, (const float *)Psi, ld, n, npts, dV, w.U, n, st));
    RS_TRY(symmetrize(w.U, n, n, st));
    RS_TRY(cholesky(w.U, n, n, 1e-14, w.status, st));
    int bad = 0;
    RS_CUDA(cudaMemcpyAsync(&bad, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    if (bad) return fail(RS_ENOTSPD, "orthonormalize: overlap matrix not positive definite (pivot %d)", bad - 1);
    RS_TRY(tri_inv(w.U, n, n, w.Ui, n, st));
    return rotate_inplace(Psi, ld, n, w.Ui, npts, dtype, st, tc);
}

// Subspace diagonalisation; eps (device, n) and w.xi receive the results.  Blocking.
int subspace_diag_impl(rs_ham *h, void *Psi, void *HPsi, int64_t ld, int n, int dtype, int nb, void *work,
                       double *eps_dev, cudaStream_t st, const TcWork &tc) {
    LaWork w(work, n);
    const int64_t npts = ham_npts(h);
    const double dV = ham_dV(h);
    const int es = dtype == RS_F64 ? 8 : 4;
    for (int b = 0; b < n; b += nb)
        RS_TRY(rs_ham_apply_block(h, (const char *)Psi + (size_t)b * es, ld, (char *)HPsi + (size_t)b * es, ld,
                                  std::min(nb, n - b), dtype, st));
    if (dtype == RS_F64)
        RS_TRY(gram<double>((const double *)Psi, ld, n, (const double *)HPsi, ld, n, npts, dV, w.S, n, st));
    else if (tc_grams(tc, n, npts))
        RS_TRY(umma_gram((const float *)Psi, ld, n, (const float *)HPsi, ld, n, npts, dV, w.S, n, tc.p, tc.err, st));
    else
        RS_TRY(gram<float>((const float *)Psi, ld, n, (const float *)HPsi, ld, n, npts, dV, w.S, n, st));
    RS_TRY(symmetrize(w.S, n, n, st));
    RS_TRY(eigh(w.S, n, n, eps_dev, w.xi, n, dtype == RS_F32 && tc.inner ? -1 : 2, w.status, w.eigw, st));
    RS_TRY(rotate_inplace(Psi, ld, n, w.xi, npts, dtype, st, tc));
    return rotate_inplace(HPsi, ld, n, w.xi, npts, dtype, st, tc);
}

}  // namespace rs

extern "C" int rs_orthonormalize(const rs_grid *g, void *Psi_dev, int64_t ld, int nst, int dtype, void *work_dev,
                                 double *Uinv_dev, void *stream) {
    if (!g || !work_dev) return fail(RS_EINVAL, "rs_orthonormalize: null argument");
    RS_TRY(check_block(Psi_dev, ld, nst, dtype));
    cudaStream_t st = (cudaStream_t)stream;
    RS_TRY(orthonormalize_impl(g->npts, g->h * g->h * g->h, Psi_dev, ld, nst, dtype, work_dev, st));
    if (Uinv_dev) {
        LaWork w(work_dev, nst);
        RS_CUDA(cudaMemcpyAsync(Uinv_dev, w.Ui, sizeof(double) * nst * nst, cudaMemcpyDeviceToDevice, st));
    }
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

extern "C" int rs_subspace_diag(rs_ham *h, void *Psi_dev, void *HPsi_dev, int64_t ld, int nst, int dtype, int nb,
                                double *eps_dev, double *xi_dev, void *work_dev, void *stream) {
    if (!h || !work_dev || !eps_dev) return fail(RS_EINVAL, "rs_subspace_diag: null argument");
    RS_TRY(check_block(Psi_dev, ld, nst, dtype));
    RS_TRY(check_block(HPsi_dev, ld, nst, dtype));
    if (nb < 1 || nb > 64 || (nb & (nb - 1))) return fail(RS_EINVAL, "rs_subspace_diag: bad nb");
    cudaStream_t st = (cudaStream_t)stream;
    RS_TRY(subspace_diag_impl(h, Psi_dev, HPsi_dev, ld, nst, dtype, nb, work_dev, eps_dev, st));
    LaWork w(work_dev, nst);
    if (xi_dev) RS_CUDA(cudaMemcpyAsync(xi_dev, w.xi, sizeof(double) * nst * nst, cudaMemcpyDeviceToDevice, st));
    int info = 0;
    RS_CUDA(cudaMemcpyAsync(&info, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    (void)info;  // FP32 Jacobi may stop at its sweep cap; the FP64 refinement that follows decides the accuracy
    return RS_OK;
}

extern "C" int64_t rs_eigh_workspace_bytes(int n) {
    if (n < 1) return -1;
    return (int64_t)eigh_work_bytes(n) + 64;
}

extern "C" int rs_eigh(const double *A_dev, int n, double *w_dev, double *V_dev, int refine, void *work_dev,
                       void *stream) {
    if (!A_dev || !w_dev || !V_dev || !work_dev || n < 2) return fail(RS_EINVAL, "rs_eigh: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int *info = reinterpret_cast<int *>((char *)work_dev + eigh_work_bytes(n));
    RS_TRY(eigh(A_dev, n, n, w_dev, V_dev, n, refine, info, work_dev, st));
    int sweeps = 0;
    RS_CUDA(cudaMemcpyAsync(&sweeps, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    if (refine == 0 && sweeps < 0) return fail(RS_ENOCONV, "rs_eigh: Jacobi sweep cap reached");
    return RS_OK;
}

/*
 * FP64 CPU oracle, native part.  TEST INFRASTRUCTURE ONLY: the product path
 * never links or calls this file; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg do.
 *
 * Plain loops, written for checkability, not speed.  Arrays are row-major.
 * Orbitals are stored point-major with the state index fastest, psi[p*nst+s]
 * (the layout of Sec. IV, Fig. 4b, for one block holding every state).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * Kohn-Sham Hamiltonian applied to nst orbitals, Eq. (3):
 *   H = -1/2 Laplacian + V_local + V_nl
 *
 * Kinetic term (Sec. V.A): star stencil of half-width m per axis,
 *   (T psi)(p) = -1/(2h^2) * sum_axis sum_{j=-m..m} c_|j| psi(p + j e_axis)
 * with psi = 0 at lattice points that are not grid points.  nbr[p][a][t]
 * holds the index of the neighbour at offset j = t-m (t != m skipped, so
 * t runs over 2m entries: j=-m..-1, 1..m) along axis a, or -1.
 *
 * Local potential (Sec. V.B): (V psi)(p) = V(p) psi(p).
 *
 * Nonlocal potential, Eq. (4) in Kleinman-Bylander form: for every atom A
 * and projector q (s, p_x, p_y, p_z)
 *   c[A,q,s] = E[A,q] * dV * sum_{p in S_A} gamma[A,q](p) psi(p,s)
 *   (V_nl psi)(p,s) = sum_{A,q : p in S_A} gamma[A,q](p) c[A,q,s]
 * computed in the paper's two parts: all integrals first, then the sum.
 * sph_off[A]..sph_off[A+1] indexes sph_idx (grid points of S_A) and
 * gam[(4*sph_off[A]) + q*len_A + i] (projector q at the i-th point).
 */
int ora_apply_h(int64_t np, int nst, int m, const int32_t *nbr, const double *cw, double h,
                const double *V, int n_atoms, const int64_t *sph_off, const int32_t *sph_idx,
                const double *gam, const double *E, double dV, const double *psi, double *hpsi)
{
    const double kin = -0.5 / (h * h);
    const int nn = 2 * m;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; ++p) {
        for (int s = 0; s < nst; ++s) {
            double acc = 3.0 * cw[0] * psi[p * nst + s];
            for (int a = 0; a < 3; ++a) {
                for (int t = 0; t < nn; ++t) {
                    int j = t < m ? t - m : t - m + 1;
                    int32_t q = nbr[(p * 3 + a) * nn + t];
                    if (q >= 0) acc += cw[j < 0 ? -j : j] * psi[(int64_t)q * nst + s];
                }
            }
            hpsi[p * nst + s] = kin * acc + V[p] * psi[p * nst + s];
        }
    }
    if (n_atoms <= 0) return 0;
    double *c = (double *)calloc((size_t)n_atoms * 4 * nst, sizeof(double));
    if (!c) return -1;
    /* part 1: projection integrals, one per (atom, projector, state) */
#pragma omp parallel for schedule(dynamic)
    for (int A = 0; A < n_atoms; ++A) {
        int64_t o = sph_off[A], len = sph_off[A + 1] - sph_off[A];
        for (int q = 0; q < 4; ++q) {
            const double *g = gam + 4 * o + q * len;
            for (int s = 0; s < nst; ++s) {
                double acc = 0.0;
                for (int64_t i = 0; i < len; ++i) acc += g[i] * psi[(int64_t)sph_idx[o + i] * nst + s];
                c[((int64_t)A * 4 + q) * nst + s] = E[A * 4 + q] * dV * acc;
            }
        }
    }
    /* part 2: multiply by the projectors and sum; atoms in sequence so that
     * overlapping spheres never write the same point concurrently */
    for (int A = 0; A < n_atoms; ++A) {
        int64_t o = sph_off[A], len = sph_off[A + 1] - sph_off[A];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < len; ++i) {
            int64_t p = sph_idx[o + i];
            for (int q = 0; q < 4; ++q) {
                double g = gam[4 * o + q * len + i];
                for (int s = 0; s < nst; ++s) hpsi[p * nst + s] += g * c[((int64_t)A * 4 + q) * nst + s];
            }
        }
    }
    free(c);
    return 0;
}

/*
 * Cholesky factorisation S = U^T U (U upper triangular), Sec. VI.
 * Textbook column-by-column form.  Returns 0, or j+1 if the j-th pivot is
 * not positive (S not positive definite).
 */
int ora_cholesky(int n, const double *S, double *U)
{
    memset(U, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double d = S[(int64_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= U[(int64_t)k * n + j] * U[(int64_t)k * n + j];
        if (!(d > 0.0)) return j + 1;
        double ujj = sqrt(d);
        U[(int64_t)j * n + j] = ujj;
        for (int i = j + 1; i < n; ++i) {
            double t = S[(int64_t)j * n + i];
            for (int k = 0; k < j; ++k) t -= U[(int64_t)k * n + j] * U[(int64_t)k * n + i];
            U[(int64_t)j * n + i] = t / ujj;
        }
    }
    return 0;
}

/* Inverse of an upper-triangular matrix by back substitution, one column
 * of the identity at a time: U X = I, X upper triangular. */
int ora_tri_inv_upper(int n, const double *U, double *X)
{
    memset(X, 0, sizeof(double) * (size_t)n * n);
    for (int col = 0; col < n; ++col) {
        for (int i = col; i >= 0; --i) {
            double t = (i == col) ? 1.0 : 0.0;
            for (int k = i + 1; k <= col; ++k) t -= U[(int64_t)i * n + k] * X[(int64_t)k * n + col];
            double d = U[(int64_t)i * n + i];
            if (d == 0.0) return -1;
            X[(int64_t)i * n + col] = t / d;
        }
    }
    return 0;
}

/*
 * Cyclic Jacobi eigenvalue algorithm for a real symmetric matrix (Jacobi
 * 1846; row-cyclic ordering with the stable rotation of Rutishauser).
 * A is n x n (overwritten).  On return w holds the eigenvalues in ascending
 * order and the columns of Vec the eigenvectors (Vec[i*n+k] = component i
 * of eigenvector k).  Returns the number of sweeps used, or -1 if max_sweeps
 * was reached before the off-diagonal norm fell below tol * ||A||_F.
 */
int ora_jacobi_eig(int n, double *A, double *w, double *Vec, int max_sweeps, double tol)
{
    double *Vt = (double *)malloc(sizeof(double) * (size_t)n * n);
    if (!Vt) return -2;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Vt[(int64_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int64_t i = 0; i < (int64_t)n * n; ++i) fro += A[i] * A[i];
    fro = sqrt(fro);
    int sweep, done = 0;
    for (sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off += A[(int64_t)i * n + j] * A[(int64_t)i * n + j];
        if (sqrt(off) <= tol * fro) { done = 1; break; }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(int64_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the rotation in the (p,q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = A[(int64_t)k * n + p], akq = A[(int64_t)k * n + q];
                    A[(int64_t)k * n + p] = c * akp - s * akq;
                    A[(int64_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(int64_t)p * n + k], aqk = A[(int64_t)q * n + k];
                    A[(int64_t)p * n + k] = c * apk - s * aqk;
                    A[(int64_t)q * n + k] = s * apk + c * aqk;
                }
                /* accumulate the rotations; row r of Vt is eigenvector r */
                for (int k = 0; k < n; ++k) {
                    double vp = Vt[(int64_t)p * n + k], vq = Vt[(int64_t)q * n + k];
                    Vt[(int64_t)p * n + k] = c * vp - s * vq;
                    Vt[(int64_t)q * n + k] = s * vp + c * vq;
                }
            }
        }
    }
    /* sort ascending (stable selection of the minimum) */
    int *ord = (int *)malloc(sizeof(int) * (size_t)n);
    char *used = (char *)calloc((size_t)n, 1);
    for (int k = 0; k < n; ++k) {
        int best = -1;
        for (int i = 0; i < n; ++i)
            if (!used[i] && (best < 0 || A[(int64_t)i * n + i] < A[(int64_t)best * n + best])) best = i;
        used[best] = 1;
        ord[k] = best;
    }
    for (int k = 0; k < n; ++k) {
        w[k] = A[(int64_t)ord[k] * n + ord[k]];
        for (int i = 0; i < n; ++i) Vec[(int64_t)i * n + k] = Vt[(int64_t)ord[k] * n + i];
    }
    free(ord);
    free(used);
    free(Vt);
    return done ? sweep : -1;
}

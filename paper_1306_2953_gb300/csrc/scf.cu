// Self-consistent field loop (Sec. III, Fig. 2) around the block
// eigensolver: each step builds the Kohn-Sham potential of the input density
// (Eq. 3: v_ext + v_H + v_xc; v_H from the FFT Poisson solver of Sec. X,
// v_xc in the local density approximation), runs a fixed number of
// eigensolver sweeps (the paper does not converge the eigenproblem inside an
// SCF step), forms the output density of Eq. 1b and mixes it by Broyden's
// scheme.  Readings (the paper names the steps, not their parameters):
//  - spin-unpolarised electrons with Fermi-Dirac occupations
//    f_k = 2 / (1 + exp((eps_k - mu) / sigma)), mu fixed by sum f_k = N_e,
//    n = sum_k f_k |phi_k|^2;
//  - LDA: Slater exchange and the Perdew-Zunger (1981) parametrisation of
//    the Ceperley-Alder correlation of the unpolarised electron gas;
//  - Broyden's second (inverse-Jacobian) update with uniform weights
//    (Broyden 1965, Srivastava 1984) in the form that equals Anderson
//    mixing: n_in' = n_in + alpha F - sum_i theta_i (dn_i + alpha dF_i),
//    F = n_out - n_in, theta minimising |F - sum theta_i dF_i|;
//  - the Mermin free energy E = sum f eps - E_H - int n v_xc + E_xc - sigma S.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "device.h"
#include "linalg.h"
#include "solver_view.h"

namespace {

constexpr double PZ_G = -0.1423, PZ_B1 = 1.0529, PZ_B2 = 0.3334;
constexpr double PZ_A = 0.0311, PZ_B = -0.048, PZ_C = 0.0020, PZ_D = -0.0116;
constexpr int MAX_HISTORY = 16;
constexpr int MAX_DOTS = 40;

// e_xc, v_xc and the Kohn-Sham potential v_ext + v_H + v_xc per point
__global__ void k_lda_potential(const double *__restrict__ n, const double *__restrict__ vext,
                                const double *__restrict__ vh, int64_t np, double *__restrict__ exc,
                                double *__restrict__ vxc, double *__restrict__ veff) {
    const double pi = 3.14159265358979323846;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const double d = n[p];
        double e = 0.0, v = 0.0;
        if (d > 1e-30) {
            const double ex = -0.75 * pow(3.0 * d / pi, 1.0 / 3.0);
            const double rs = pow(3.0 / (4.0 * pi * d), 1.0 / 3.0);
            double ec, vc;
            if (rs >= 1.0) {
                const double sq = sqrt(rs), den = 1.0 + PZ_B1 * sq + PZ_B2 * rs;
                ec = PZ_G / den;
                vc = ec * (1.0 + 7.0 / 6.0 * PZ_B1 * sq + 4.0 / 3.0 * PZ_B2 * rs) / den;
            } else {
                const double lr = log(rs);
                ec = PZ_A * lr + PZ_B + PZ_C * rs * lr + PZ_D * rs;
                vc = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * rs * lr + (2.0 * PZ_D - PZ_C) / 3.0 * rs;
            }
            e = ex + ec;
            v = 4.0 / 3.0 * ex + vc;
        }
        exc[p] = e;
        vxc[p] = v;
        veff[p] = vext[p] + vh[p] + v;
    }
}

// n[p] = sum_k f_k psi[p][k]^2
template <typename T>
__global__ void k_density(const T *__restrict__ psi, int nst, const double *__restrict__ f, int64_t np,
                          double *__restrict__ n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const T *row = psi + p * nst;
        double acc = 0.0;
        for (int k = 0; k < nst; ++k) {
            const double v = (double)row[k];
            acc += __ldg(f + k) * v * v;
        }
        n[p] = acc;
    }
}

__global__ void k_weight_by_norm(double *f, const double *norm2, double dV, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) f[k] /= dV * norm2[k];
}

__global__ void k_diff(const double *__restrict__ a, const double *__restrict__ b, int64_t np, double *__restrict__ c) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x)
        c[p] = a[p] - b[p];
}

struct DotList {
    const double *a[MAX_DOTS];
    const double *b[MAX_DOTS];
    int n;
};

// out[q] = sum_p a_q[p] b_q[p] (out zeroed by the caller)
__global__ void k_dots(DotList d, int64_t np, double *out) {
    __shared__ double red[256];
    for (int q = 0; q < d.n; ++q) {
        double acc = 0.0;
        for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x)
            acc += d.a[q][p] * d.b[q][p];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(out + q, red[0]);
        __syncthreads();
    }
}

struct MixTerms {
    const double *dn[MAX_HISTORY];
    const double *dF[MAX_HISTORY];
    double theta[MAX_HISTORY];
    int m;
};

// out = n + alpha F - sum_i theta_i (dn_i + alpha dF_i)
__global__ void k_mix(const double *__restrict__ n, const double *__restrict__ F, double alpha, MixTerms t, int64_t np,
                      double *__restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        double v = n[p] + alpha * F[p];
        for (int i = 0; i < t.m; ++i) v -= t.theta[i] * (t.dn[i][p] + alpha * t.dF[i][p]);
        out[p] = v;
    }
}

// A x = b by Gaussian elimination with partial pivoting (A row-major m x m)
bool solve_small(std::vector<double> A, std::vector<double> b, int m, std::vector<double> &x) {
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(A[r * m + c]) > std::fabs(A[piv * m + c])) piv = r;
        if (A[piv * m + c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < m; ++k) std::swap(A[c * m + k], A[piv * m + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < m; ++r) {
            const double l = A[r * m + c] / A[c * m + c];
            for (int k = c; k < m; ++k) A[r * m + k] -= l * A[c * m + k];
            b[r] -= l * b[c];
        }
    }
    x.assign(m, 0.0);
    for (int r = m - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < m; ++k) s -= A[r * m + k] * x[k];
        x[r] = s / A[r * m + r];
    }
    return true;
}

unsigned grid1d(int64_t np) { return (unsigned)std::min<int64_t>((np + 255) / 256, 152 * 8); }

}  // namespace

struct rs_scf {
    rs_solver *s = nullptr;
    rs_poisson *poisson = nullptr;
    rs_scf_cfg cfg{};
    int64_t np = 0;
    double dV = 0;
    rs::DevBuf vext, n_in, n_out, F, vh, vxc, exc, veff, fdev, prev_n, prev_F, hist, dots, eps64, norm2;
    std::vector<int> order;    // history slots, oldest first
    bool have_prev = false;
    std::vector<double> f;
    double mu = 0, residual = 0, energy = 0;
    int iterations = 0;
    ~rs_scf() {
        if (poisson) rs_poisson_destroy(poisson);
    }
};

using rs::fail;

extern "C" int rs_scf_create(rs_solver *s, const rs_grid *g, const double *v_ext_host, const double *n0_host,
                             const rs_scf_cfg *cfg, rs_scf **out) {
    if (!s || !g || !v_ext_host || !n0_host || !cfg || !out) return fail(RS_EINVAL, "rs_scf_create: null argument");
    *out = nullptr;
    const rs_scf_cfg c = *cfg;
    rs::SolverView v;
    rs::solver_view(s, &v);
    if (v.npts != g->npts) return fail(RS_EINVAL, "rs_scf_create: grid and solver differ");
    if (!(c.n_electrons > 0) || c.n_electrons > 2.0 * v.nst || !(c.sigma > 0) || !(c.alpha > 0) || c.history < 0 ||
        c.history > MAX_HISTORY || c.sweeps < 1)
        return fail(RS_EINVAL, "rs_scf_create: bad configuration");
    rs_scf *S = new (std::nothrow) rs_scf;
    if (!S) return fail(RS_ENOMEM, "host allocation failed");
    auto bail = [&](int rc) {
        delete S;
        return rc;
    };
    S->s = s;
    S->cfg = c;
    S->np = v.npts;
    S->dV = v.dV;
    const size_t vb = sizeof(double) * (size_t)S->np;
    int rc;
    if ((rc = rs_poisson_create(g, &S->poisson)) || (rc = S->vext.upload(v_ext_host, vb)) ||
        (rc = S->n_in.upload(n0_host, vb)) || (rc = S->n_out.alloc(vb)) || (rc = S->F.alloc(vb)) ||
        (rc = S->vh.alloc(vb)) || (rc = S->vxc.alloc(vb)) || (rc = S->exc.alloc(vb)) || (rc = S->veff.alloc(vb)) ||
        (rc = S->fdev.alloc(sizeof(double) * v.nst)) || (rc = S->prev_n.alloc(vb)) || (rc = S->prev_F.alloc(vb)) ||
        (rc = S->hist.alloc(2 * vb * (size_t)std::max(c.history, 1))) || (rc = S->dots.alloc(sizeof(double) * MAX_DOTS)))
        return bail(rc);
    *out = S;
    return RS_OK;
}

static int dots(rs_scf *S, const DotList &d, std::vector<double> &out, cudaStream_t st) {
    RS_CUDA(cudaMemsetAsync(S->dots.p, 0, sizeof(double) * d.n, st));
    k_dots<<<grid1d(S->np), 256, 0, st>>>(d, S->np, S->dots.as<double>());
    RS_LAUNCH_CHECK();
    out.resize(d.n);
    RS_CUDA(cudaMemcpyAsync(out.data(), S->dots.p, sizeof(double) * d.n, cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

extern "C" int rs_scf_step(rs_scf *S, double *residual, double *energy, void *stream) {
    if (!S) return fail(RS_EINVAL, "rs_scf_step: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const rs_scf_cfg &c = S->cfg;
    const int64_t np = S->np;
    // Kohn-Sham potential of the input density
    RS_TRY(rs_poisson_solve(S->poisson, S->n_in.as<double>(), S->vh.as<double>(), st));
    k_lda_potential<<<grid1d(np), 256, 0, st>>>(S->n_in.as<double>(), S->vext.as<double>(), S->vh.as<double>(), np,
                                                S->exc.as<double>(), S->vxc.as<double>(), S->veff.as<double>());
    RS_LAUNCH_CHECK();
    RS_TRY(rs_solver_set_potential(S->s, S->veff.as<double>(), st));
    for (int k = 0; k < c.sweeps; ++k) RS_TRY(rs_eigensolver_step(S->s, nullptr, nullptr, nullptr, st));
    // occupations (host bisection on the eigenvalues) and the output density;
    // FP32 solvers: the eigenvalues of the FP64 Rayleigh-Ritz of their
    // subspace (H applied in FP64), so that the occupations and the band
    // energy carry no FP32 rounding of H
    rs::SolverView v;
    rs::solver_view(S->s, &v);
    const double *eig = v.eig;
    if (v.dtype == RS_F32) {
        if (!S->eps64.p) RS_TRY(S->eps64.alloc(sizeof(double) * v.nst));
        RS_TRY(rs_solver_rayleigh_ritz_f64(S->s, S->eps64.as<double>(), st));
        eig = S->eps64.as<double>();
    }
    std::vector<double> eps(v.nst);
    RS_CUDA(cudaMemcpyAsync(eps.data(), eig, sizeof(double) * v.nst, cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    const double emin = *std::min_element(eps.begin(), eps.end()), emax = *std::max_element(eps.begin(), eps.end());
    auto fd = [&](double mu, std::vector<double> &f) {
        double sum = 0;
        f.resize(eps.size());
        for (size_t k = 0; k < eps.size(); ++k) {
            const double x = std::min(700.0, std::max(-700.0, (eps[k] - mu) / c.sigma));
            f[k] = 2.0 / (1.0 + std::exp(x));
            sum += f[k];
        }
        return sum;
    };
    double lo = emin - 50 * c.sigma, hi = emax + 50 * c.sigma;
    std::vector<double> f;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (fd(mid, f) < c.n_electrons) lo = mid;
        else hi = mid;
    }
    S->mu = 0.5 * (lo + hi);
    fd(S->mu, f);
    S->f = f;
    RS_CUDA(cudaMemcpyAsync(S->fdev.p, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice, st));
    // each orbital's weight divided by its norm <phi_k|phi_k>, summed in FP64:
    // FP32 orbitals are normalised through the tensor-core overlap, whose
    // FP32 accumulation leaves norms off one by up to ~1e-6, enough to change
    // the total charge (and every eigenvalue, through v_H) by ~1e-4
    if (!S->norm2.p) RS_TRY(S->norm2.alloc(sizeof(double) * v.nst));
    for (int k0 = 0; k0 < v.nst; k0 += 256) {
        const int nc = std::min(256, v.nst - k0);
        const int64_t es = v.dtype == RS_F64 ? 8 : 4;
        const void *col = (const char *)v.psi + k0 * es;
        RS_TRY(rs::coldots(v.dtype, col, v.nst, col, v.nst, nc, np, S->norm2.as<double>() + k0, st));
    }
    k_weight_by_norm<<<(v.nst + 255) / 256, 256, 0, st>>>(S->fdev.as<double>(), S->norm2.as<double>(), S->dV, v.nst);
    RS_LAUNCH_CHECK();
    if (v.dtype == RS_F64)
        k_density<double><<<grid1d(np), 256, 0, st>>>((const double *)v.psi, v.nst, S->fdev.as<double>(), np,
                                                      S->n_out.as<double>());
    else
        k_density<float><<<grid1d(np), 256, 0, st>>>((const float *)v.psi, v.nst, S->fdev.as<double>(), np,
                                                     S->n_out.as<double>());
    k_diff<<<grid1d(np), 256, 0, st>>>(S->n_out.as<double>(), S->n_in.as<double>(), np, S->F.as<double>());
    RS_LAUNCH_CHECK();
    // residual and energy terms
    {
        DotList d{};
        const double *ni = S->n_in.as<double>();
        d.a[0] = S->F.as<double>(), d.b[0] = S->F.as<double>();
        d.a[1] = ni, d.b[1] = S->vh.as<double>();
        d.a[2] = ni, d.b[2] = S->vxc.as<double>();
        d.a[3] = ni, d.b[3] = S->exc.as<double>();
        d.n = 4;
        std::vector<double> r;
        RS_TRY(dots(S, d, r, st));
        double band = 0, ent = 0;
        for (size_t k = 0; k < f.size(); ++k) {
            band += f[k] * eps[k];
            const double x = std::min(std::max(f[k] / 2.0, 1e-300), 1.0 - 1e-16);
            ent += -2.0 * (x * std::log(x) + (1.0 - x) * std::log1p(-x));
        }
        S->residual = std::sqrt(S->dV * r[0]);
        S->energy = band - 0.5 * S->dV * r[1] - S->dV * r[2] + S->dV * r[3] - c.sigma * ent;
        if (!std::isfinite(S->residual) || !std::isfinite(S->energy))
            return fail(RS_ENAN, "rs_scf_step: non-finite density residual or energy");
    }
    // Broyden mixing: history (dn, dF) of the last `history` steps
    const size_t vb = sizeof(double) * (size_t)np;
    double *hist = S->hist.as<double>();
    auto dn_of = [&](int slot) { return hist + (size_t)(2 * slot) * np; };
    auto dF_of = [&](int slot) { return hist + (size_t)(2 * slot + 1) * np; };
    if (S->have_prev && c.history > 0) {
        int slot;
        if ((int)S->order.size() < c.history) {
            slot = (int)S->order.size();
        } else {
            slot = S->order.front();
            S->order.erase(S->order.begin());
        }
        S->order.push_back(slot);
        k_diff<<<grid1d(np), 256, 0, st>>>(S->n_in.as<double>(), S->prev_n.as<double>(), np, dn_of(slot));
        k_diff<<<grid1d(np), 256, 0, st>>>(S->F.as<double>(), S->prev_F.as<double>(), np, dF_of(slot));
        RS_LAUNCH_CHECK();
    }
    RS_CUDA(cudaMemcpyAsync(S->prev_n.p, S->n_in.p, vb, cudaMemcpyDeviceToDevice, st));
    RS_CUDA(cudaMemcpyAsync(S->prev_F.p, S->F.p, vb, cudaMemcpyDeviceToDevice, st));
    S->have_prev = true;
    MixTerms t{};
    const int m = (int)S->order.size();
    if (m > 0) {
        // G_ij = <dF_i|dF_j>, rhs_i = <dF_i|F> (the grid weight dV cancels)
        DotList d{};
        for (int i = 0; i < m; ++i)
            for (int j = i; j < m; ++j) {
                d.a[d.n] = dF_of(S->order[i]), d.b[d.n] = dF_of(S->order[j]);
                ++d.n;
            }
        std::vector<double> g, r;
        RS_TRY(dots(S, d, g, st));
        DotList e{};
        for (int i = 0; i < m; ++i) e.a[e.n] = dF_of(S->order[i]), e.b[e.n] = S->F.as<double>(), ++e.n;
        RS_TRY(dots(S, e, r, st));
        std::vector<double> G((size_t)m * m), theta;
        for (int i = 0, q = 0; i < m; ++i)
            for (int j = i; j < m; ++j, ++q) G[(size_t)i * m + j] = G[(size_t)j * m + i] = g[q];
        if (!solve_small(G, r, m, theta)) return fail(RS_ENAN, "rs_scf_step: singular Broyden system");
        for (int i = 0; i < m; ++i) {
            t.dn[i] = dn_of(S->order[i]);
            t.dF[i] = dF_of(S->order[i]);
            t.theta[i] = theta[i];
        }
        t.m = m;
    }
    k_mix<<<grid1d(np), 256, 0, st>>>(S->n_in.as<double>(), S->F.as<double>(), c.alpha, t, np, S->n_out.as<double>());
    RS_LAUNCH_CHECK();
    RS_CUDA(cudaMemcpyAsync(S->n_in.p, S->n_out.p, vb, cudaMemcpyDeviceToDevice, st));
    RS_CUDA(cudaStreamSynchronize(st));
    ++S->iterations;
    if (residual) *residual = S->residual;
    if (energy) *energy = S->energy;
    return RS_OK;
}

extern "C" int rs_scf_state(rs_scf *S, double *n_in_dev, double *occupations_host, double *mu, int *iterations) {
    if (!S) return fail(RS_EINVAL, "rs_scf_state: null handle");
    if (n_in_dev) RS_CUDA(cudaMemcpy(n_in_dev, S->n_in.p, sizeof(double) * (size_t)S->np, cudaMemcpyDeviceToDevice));
    if (occupations_host) std::copy(S->f.begin(), S->f.end(), occupations_host);
    if (mu) *mu = S->mu;
    if (iterations) *iterations = S->iterations;
    return RS_OK;
}

extern "C" int rs_scf_destroy(rs_scf *S) {
    delete S;
    return RS_OK;
}

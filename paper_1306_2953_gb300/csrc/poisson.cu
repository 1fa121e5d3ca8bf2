// Hartree potential by fast Fourier transforms (Sec. X; Eq. 2, the Poisson
// equation lap V_H = -4 pi n), the paper's steps on the GPU:
//   1. the density is copied from the grid to a cube (zero elsewhere);
//   2. forward 3-D FFT;
//   3. multiplication by the Coulomb-interaction kernel;
//   4. inverse 3-D FFT;
//   5. the potential is copied back to the grid.
// Free boundary conditions: an enlarged cube and the spherical-cutoff kernel
// of Rozzi et al. (2006), the Coulomb potential cut off at r = R_c,
//   v(G) = 4 pi (1 - cos(|G| R_c)) / |G|^2,   v(0) = 2 pi R_c^2,
// with R_c = D + h (D: the diagonal of the grid's bounding box) and N_a
// points along axis a, the smallest 2^p 3^q >= extent_a + ceil(R_c / h) + 1,
// so that no periodic image of the density lies within R_c of it.
//
// FFT: complex FP64, one kernel launch per axis and direction.  A CTA
// transforms LN lines of one axis held in shared memory: it loads them
// (for the two strided axes the LN lines are adjacent along the contiguous
// axis, so every row of the tile is one contiguous LN * 16-byte segment),
// runs the Stockham autosort passes of radix 3, 4 and 2 (Govindaraju et al.
// 2008 formulation: pass with radix R and span Ns reads R inputs N/R apart,
// twiddles them by exp(-+2 pi i r (j mod Ns) / (Ns R)), takes an R-point
// DFT and writes R outputs Ns apart), and stores the lines back.  The
// twiddles come from a table of exp(2 pi i m / N), m < N, staged in shared
// memory (the angle of input r of butterfly j is m = r (j mod Ns) N / (Ns R)):
// no transcendental function runs in the passes, which matters on GB300,
// whose FP64 units are a small fraction of its FP32 ones.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "device.h"

namespace {

constexpr int LN = 8;          // lines per CTA
constexpr int FFT_NT = 256;
constexpr int MAX_N = 768;     // largest axis length (two LN-line buffers and the table fit in shared memory)

struct Cplx {
    double x, y;
};
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ Cplx cadd(Cplx a, Cplx b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ Cplx csub(Cplx a, Cplx b) { return {a.x - b.x, a.y - b.y}; }

struct Radices {
    int r[24];
    int n;
};

// One axis of the 3-D transform.  Element j of line l of the CTA's tile is at
// base + l * ls + j * es; the tile's base: axis 2 (contiguous): lines are
// whole rows, base = (blockIdx.x * LN) * N, ls = N, es = 1; axes 0 and 1:
// lines adjacent along axis 2, base from (outer, i2 block), ls = 1.
// sign = -1 forward, +1 inverse (unnormalised).
__global__ void __launch_bounds__(FFT_NT) k_fft_axis(Cplx *__restrict__ data, int N, int64_t es,
                                                      int64_t nlines, int n2, int64_t outer_stride, int axis,
                                                      Radices rad, int sign, const Cplx *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char fsm[];
    Cplx *A = reinterpret_cast<Cplx *>(fsm);
    Cplx *B = A + LN * N;
    Cplx *T = B + LN * N;   // exp(2 pi i m / N)
    // tile base and the number of valid lines
    int64_t base;
    int nl;
    if (axis == 2) {
        const int64_t l0 = (int64_t)blockIdx.x * LN;
        base = l0 * N;
        nl = nlines - l0 < LN ? (int)(nlines - l0) : LN;
    } else {
        // lines indexed (outer, i2): outer = blockIdx.y, i2 block = blockIdx.x
        const int i20 = blockIdx.x * LN;
        base = (int64_t)blockIdx.y * outer_stride + i20;
        nl = min(LN, n2 - i20);
    }
    if (nl <= 0) return;
    for (int m = threadIdx.x; m < N; m += FFT_NT) T[m] = tw[m];
    // load: smem layout [line][j]
    if (axis == 2) {
        for (int e = threadIdx.x; e < nl * N; e += FFT_NT) A[e] = data[base + e];
    } else {
        for (int e = threadIdx.x; e < nl * N; e += FFT_NT) {
            const int j = e / nl, l = e - j * nl;     // consecutive threads: consecutive lines of one row
            A[l * N + j] = data[base + (int64_t)j * es + l];
        }
    }
    __syncthreads();
    Cplx *x = A, *y = B;
    int Ns = 1;
    const double s3 = 0.86602540378443864676;   // sin(2 pi / 3)
    for (int p = 0; p < rad.n; ++p) {
        const int R = rad.r[p], M = N / R, step = N / (Ns * R);
        for (int e = threadIdx.x; e < nl * M; e += FFT_NT) {
            const int l = e / M, j = e - l * M;
            const Cplx *xl = x + l * N;
            Cplx *yl = y + l * N;
            const int k = j % Ns;
            const int out = (j / Ns) * Ns * R + k;
            // input r twiddled by exp(sign 2 pi i r k / (Ns R)) = T[r k step] (conjugated for sign < 0)
            auto tw_r = [&](int r) {
                const Cplx w = T[r * k * step];
                return Cplx{w.x, (double)sign * w.y};
            };
            if (R == 2) {
                Cplx v0 = xl[j], v1 = xl[j + M];
                if (k) v1 = cmul(v1, tw_r(1));
                yl[out] = cadd(v0, v1);
                yl[out + Ns] = csub(v0, v1);
            } else if (R == 4) {
                Cplx v0 = xl[j], v1 = xl[j + M], v2 = xl[j + 2 * M], v3 = xl[j + 3 * M];
                if (k) {
                    v1 = cmul(v1, tw_r(1));
                    v2 = cmul(v2, tw_r(2));
                    v3 = cmul(v3, tw_r(3));
                }
                const Cplx a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = csub(v1, v3);
                const Cplx wd = {-(double)sign * d.y, (double)sign * d.x};   // sign i (v1 - v3)
                yl[out] = cadd(a, c);
                yl[out + Ns] = cadd(b, wd);
                yl[out + 2 * Ns] = csub(a, c);
                yl[out + 3 * Ns] = csub(b, wd);
            } else {
                Cplx v0 = xl[j], v1 = xl[j + M], v2 = xl[j + 2 * M];
                if (k) {
                    v1 = cmul(v1, tw_r(1));
                    v2 = cmul(v2, tw_r(2));
                }
                const Cplx t1 = cadd(v1, v2);
                const Cplx t2 = {v0.x - 0.5 * t1.x, v0.y - 0.5 * t1.y};
                // i * sign * sin(2 pi / 3) * (v1 - v2)
                const Cplx d = csub(v1, v2);
                const Cplx t3 = {-(double)sign * s3 * d.y, (double)sign * s3 * d.x};
                yl[out] = cadd(v0, t1);
                yl[out + Ns] = cadd(t2, t3);
                yl[out + 2 * Ns] = csub(t2, t3);
            }
        }
        __syncthreads();
        Cplx *t = x;
        x = y;
        y = t;
        Ns *= R;
    }
    if (axis == 2) {
        for (int e = threadIdx.x; e < nl * N; e += FFT_NT) data[base + e] = x[e];
    } else {
        for (int e = threadIdx.x; e < nl * N; e += FFT_NT) {
            const int j = e / nl, l = e - j * nl;
            data[base + (int64_t)j * es + l] = x[l * N + j];
        }
    }
}

__global__ void k_scatter(const double *__restrict__ n, const int32_t *__restrict__ cidx, int64_t npts,
                          Cplx *__restrict__ cube) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x)
        cube[cidx[p]] = {n[p], 0.0};
}

// v(G) on the cube: G_a = 2 pi f_a / (N_a h), f_a the signed frequency of
// index i_a (computed once per plan)
__global__ void k_kernel_values(double *__restrict__ vg, int n0, int n1, int n2, double h, double rc) {
    const int64_t tot = (int64_t)n0 * n1 * n2;
    const double tp = 2.0 * 3.14159265358979323846;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(e % n2), i1 = (int)((e / n2) % n1), i0 = (int)(e / ((int64_t)n1 * n2));
        const int f0 = i0 < (n0 + 1) / 2 ? i0 : i0 - n0, f1 = i1 < (n1 + 1) / 2 ? i1 : i1 - n1,
                  f2 = i2 < (n2 + 1) / 2 ? i2 : i2 - n2;
        const double g0 = tp * f0 / (n0 * h), g1 = tp * f1 / (n1 * h), g2 = tp * f2 / (n2 * h);
        const double G2 = g0 * g0 + g1 * g1 + g2 * g2;
        vg[e] = e == 0 ? 2.0 * 3.14159265358979323846 * rc * rc : 2.0 * tp * (1.0 - cos(sqrt(G2) * rc)) / G2;
    }
}

__global__ void k_kernel_mul(Cplx *__restrict__ cube, const double *__restrict__ vg, int64_t tot) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = vg[e];
        const Cplx c = cube[e];
        cube[e] = {c.x * v, c.y * v};
    }
}

__global__ void k_gather(const Cplx *__restrict__ cube, const int32_t *__restrict__ cidx, int64_t npts, double scale,
                         double *__restrict__ v) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x)
        v[p] = cube[cidx[p]].x * scale;
}

int smooth_size(int n) {
    int best = -1;
    for (int64_t p2 = 1; p2 < 2 * (int64_t)n + 2; p2 *= 2)
        for (int64_t p3 = p2; p3 < 2 * (int64_t)n + 2; p3 *= 3)
            if (p3 >= n && (best < 0 || p3 < best)) best = (int)p3;
    return best;
}

Radices radices(int n) {
    Radices r{};
    while (n % 3 == 0) {
        r.r[r.n++] = 3;
        n /= 3;
    }
    while (n % 4 == 0) {
        r.r[r.n++] = 4;
        n /= 4;
    }
    while (n % 2 == 0) {
        r.r[r.n++] = 2;
        n /= 2;
    }
    return r;
}

}  // namespace

struct rs_poisson {
    int64_t npts = 0;
    int n[3] = {0, 0, 0};
    double h = 0, rc = 0;
    rs::DevBuf cube, cidx, vg, tw[3];   // vg: v(G) per cube element; tw[a]: exp(2 pi i m / n[a]), m < n[a]
};

using rs::fail;

extern "C" int rs_poisson_create(const rs_grid *g, rs_poisson **out) {
    if (!g || !out) return fail(RS_EINVAL, "rs_poisson_create: null argument");
    *out = nullptr;
    if (g->npts < 1) return fail(RS_EINVAL, "rs_poisson_create: empty grid");
    int32_t lo[3], hi[3];
    for (int d = 0; d < 3; ++d) lo[d] = hi[d] = g->ijk[d];
    for (int64_t p = 0; p < g->npts; ++p)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], g->ijk[3 * p + d]);
            hi[d] = std::max(hi[d], g->ijk[3 * p + d]);
        }
    double D2 = 0;
    for (int d = 0; d < 3; ++d) D2 += (double)(hi[d] - lo[d]) * (double)(hi[d] - lo[d]);
    const double rc = g->h * std::sqrt(D2) + g->h;
    rs_poisson *P = new (std::nothrow) rs_poisson;
    if (!P) return fail(RS_ENOMEM, "host allocation failed");
    P->npts = g->npts;
    P->h = g->h;
    P->rc = rc;
    int64_t tot = 1;
    for (int d = 0; d < 3; ++d) {
        P->n[d] = smooth_size((hi[d] - lo[d]) + (int)std::ceil(rc / g->h) + 1);
        if (P->n[d] > MAX_N) {
            delete P;
            return fail(RS_EINVAL, "rs_poisson_create: cube of %d points along an axis exceeds %d", P->n[d], MAX_N);
        }
        tot *= P->n[d];
    }
    if (tot > INT32_MAX) {
        delete P;
        return fail(RS_EINVAL, "rs_poisson_create: cube too large");
    }
    std::vector<int32_t> idx((size_t)g->npts);
    for (int64_t p = 0; p < g->npts; ++p)
        idx[p] = (int32_t)(((int64_t)(g->ijk[3 * p] - lo[0]) * P->n[1] + (g->ijk[3 * p + 1] - lo[1])) * P->n[2] +
                           (g->ijk[3 * p + 2] - lo[2]));
    int rc2;
    if ((rc2 = P->cidx.upload(idx.data(), idx.size() * sizeof(int32_t))) ||
        (rc2 = P->cube.alloc((size_t)tot * sizeof(Cplx))) || (rc2 = P->vg.alloc((size_t)tot * sizeof(double)))) {
        delete P;
        return rc2;
    }
    k_kernel_values<<<152 * 16, 256>>>(P->vg.as<double>(), P->n[0], P->n[1], P->n[2], P->h, P->rc);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        delete P;
        return fail(RS_ECUDA, "rs_poisson_create: kernel table failed");
    }
    for (int d = 0; d < 3; ++d) {
        std::vector<Cplx> t((size_t)P->n[d]);
        const double tp = 2.0 * 3.14159265358979323846;
        for (int m = 0; m < P->n[d]; ++m) t[m] = {std::cos(tp * m / P->n[d]), std::sin(tp * m / P->n[d])};
        if ((rc2 = P->tw[d].upload(t.data(), t.size() * sizeof(Cplx)))) {
            delete P;
            return rc2;
        }
    }
    *out = P;
    return RS_OK;
}

extern "C" int rs_poisson_info(const rs_poisson *P, int32_t shape[3], double *r_cut, int64_t *cube_bytes) {
    if (!P) return fail(RS_EINVAL, "rs_poisson_info: null handle");
    for (int d = 0; d < 3 && shape; ++d) shape[d] = P->n[d];
    if (r_cut) *r_cut = P->rc;
    if (cube_bytes) *cube_bytes = (int64_t)P->n[0] * P->n[1] * P->n[2] * (int64_t)sizeof(Cplx);
    return RS_OK;
}

static int fft3(rs_poisson *P, int sign, cudaStream_t st) {
    Cplx *c = P->cube.as<Cplx>();
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    for (int axis = 2; axis >= 0; --axis) {
        const int N = P->n[axis];
        const Radices rad = radices(N);
        const Cplx *tw = P->tw[axis].as<Cplx>();
        const size_t smem = (2 * (size_t)LN + 1) * N * sizeof(Cplx);
        RS_TRY(rs::smem_optin((const void *)k_fft_axis, smem));
        if (axis == 2) {
            const int64_t nlines = (int64_t)n0 * n1;
            k_fft_axis<<<(unsigned)((nlines + LN - 1) / LN), FFT_NT, smem, st>>>(c, N, 1, nlines, n2, 0, 2, rad, sign, tw);
        } else if (axis == 1) {
            // lines (i0, i2), elements stride n2; outer = i0
            k_fft_axis<<<dim3((unsigned)((n2 + LN - 1) / LN), (unsigned)n0), FFT_NT, smem, st>>>(
                c, N, n2, 0, n2, (int64_t)n1 * n2, 1, rad, sign, tw);
        } else {
            // lines (i1, i2), elements stride n1 n2; outer = i1
            k_fft_axis<<<dim3((unsigned)((n2 + LN - 1) / LN), (unsigned)n1), FFT_NT, smem, st>>>(
                c, N, (int64_t)n1 * n2, 0, n2, (int64_t)n2, 0, rad, sign, tw);
        }
        RS_LAUNCH_CHECK();
    }
    return RS_OK;
}

extern "C" int rs_poisson_solve(rs_poisson *P, const double *n_dev, double *vh_dev, void *stream) {
    if (!P || !n_dev || !vh_dev) return fail(RS_EINVAL, "rs_poisson_solve: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t tot = (int64_t)P->n[0] * P->n[1] * P->n[2];
    RS_CUDA(cudaMemsetAsync(P->cube.p, 0, (size_t)tot * sizeof(Cplx), st));
    const unsigned pb = (unsigned)std::min<int64_t>((P->npts + 255) / 256, 152 * 16);
    k_scatter<<<pb, 256, 0, st>>>(n_dev, P->cidx.as<int32_t>(), P->npts, P->cube.as<Cplx>());
    RS_LAUNCH_CHECK();
    RS_TRY(fft3(P, -1, st));
    k_kernel_mul<<<152 * 16, 256, 0, st>>>(P->cube.as<Cplx>(), P->vg.as<double>(), tot);
    RS_LAUNCH_CHECK();
    RS_TRY(fft3(P, +1, st));
    k_gather<<<pb, 256, 0, st>>>(P->cube.as<Cplx>(), P->cidx.as<int32_t>(), P->npts, 1.0 / (double)tot, vh_dev);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

extern "C" int rs_poisson_destroy(rs_poisson *P) {
    delete P;
    return RS_OK;
}

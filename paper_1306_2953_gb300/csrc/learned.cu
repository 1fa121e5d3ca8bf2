// Learned preconditioner: training targets, a small 3-D convolutional
// network, its training kernels and its inference inside the eigensolver.
// None of this is in the paper (its preconditioner is the filter of
// Sec. III); the definitions are:
//
//  Target generator: conjugate gradients for exactly n_iter iterations from
//  x = 0 on (-1/2 Lap + sigma) x = r, one system per column, with the
//  operator applied by the H psi kernels of a Hamiltonian built with
//  V = sigma and no projectors.
//
//  Network: y = L3(relu(L2(relu(L1(xhat))))), 3^3 bias-free cross-
//  correlations 1 -> 8 -> 8 -> 1 on the lattice, every layer's output zero
//  off the grid, xhat = r / rms(r) stored in BF16, weights used in BF16
//  (rounded from an FP32 master copy), FP32 accumulation; K r = rms(r) y.
//  Weights: one FP32 array of 2160 values, [8][1][27] | [8][8][27] |
//  [1][8][27], tap t = 9 (a+1) + 3 (b+1) + (c+1) for the offset (a, b, c)
//  along map axes (0, 1, 2).
//
//  Training: tiles of D^3 lattice points (a 16^3 interior plus 3 points of
//  halo) cut around random grid points of (residual, CG solution) pairs;
//  loss = mean squared error over interior grid points; Adam
//  (lr, beta = (0.9, 0.999), eps = 1e-8) on the FP32 master weights.
#include <algorithm>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "device.h"
#include "ham.h"
#include "learned.h"
#include "linalg.h"

namespace rs {

constexpr int NC = 8;                        // hidden channels
constexpr int W1_OFF = 0, W2_OFF = NC * 27, W3_OFF = NC * 27 + NC * NC * 27, W_TOTAL = W3_OFF + NC * 27;
static_assert(W_TOTAL == 2160, "weight layout");

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ------------------------------------------------------------------- CG ---

template <typename T>
__global__ void k_cg_init(const T *__restrict__ B, int64_t ldb, T *__restrict__ X, int64_t ldx, T *__restrict__ R,
                          T *__restrict__ P, int n, int64_t npts) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = t / n;
    const int k = (int)(t % n);
    if (p >= npts) return;
    const T b = B[p * ldb + k];
    X[p * ldx + k] = 0;
    R[p * n + k] = b;
    P[p * n + k] = b;
}

// X += alpha P, R -= alpha AP with alpha = rr / pAp per column
template <typename T>
__global__ void k_cg_update1(T *__restrict__ X, int64_t ldx, T *__restrict__ R, const T *__restrict__ P,
                             const T *__restrict__ AP, const double *__restrict__ rr, const double *__restrict__ pap,
                             int n, int64_t npts) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = t / n;
    const int k = (int)(t % n);
    if (p >= npts) return;
    const T a = pap[k] != 0.0 ? (T)(rr[k] / pap[k]) : T(0);
    X[p * ldx + k] += a * P[p * n + k];
    R[p * n + k] -= a * AP[p * n + k];
}

// P = R + beta P with beta = rr_new / rr per column
template <typename T>
__global__ void k_cg_update2(const T *__restrict__ R, T *__restrict__ P, const double *__restrict__ rr,
                             const double *__restrict__ rr_new, int n, int64_t npts) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = t / n;
    const int k = (int)(t % n);
    if (p >= npts) return;
    const T b = rr[k] != 0.0 ? (T)(rr_new[k] / rr[k]) : T(0);
    P[p * n + k] = R[p * n + k] + b * P[p * n + k];
}

__global__ void k_copy_d(const double *a, double *b, int n) {
    if (threadIdx.x < n) b[threadIdx.x] = a[threadIdx.x];
}

int64_t cg_workspace_bytes(int64_t npts, int ncols, int dtype) {
    const int es = dtype == RS_F64 ? 8 : 4;
    return 3 * npts * ncols * es + 4 * 64 * 8 + 256;
}

template <typename T>
static int cg_t(rs_ham *h, const T *B, int64_t ldb, T *X, int64_t ldx, int n, int n_iter, void *work, cudaStream_t st) {
    const int64_t np = ham_npts(h);
    T *R = reinterpret_cast<T *>(work);
    T *P = R + np * n;
    T *AP = P + np * n;
    double *rr = reinterpret_cast<double *>(AP + np * n);
    double *pap = rr + 64, *rrn = pap + 64;
    const int dt = sizeof(T) == 8 ? RS_F64 : RS_F32;
    const unsigned blocks = (unsigned)((np * n + 255) / 256);
    k_cg_init<T><<<blocks, 256, 0, st>>>(B, ldb, X, ldx, R, P, n, np);
    RS_LAUNCH_CHECK();
    RS_TRY(coldots(dt, R, n, R, n, n, np, rr, st));
    for (int it = 0; it < n_iter; ++it) {
        RS_TRY(rs_ham_apply_block(h, P, n, AP, n, n, dt, st));
        RS_TRY(coldots(dt, P, n, AP, n, n, np, pap, st));
        k_cg_update1<T><<<blocks, 256, 0, st>>>(X, ldx, R, P, AP, rr, pap, n, np);
        RS_LAUNCH_CHECK();
        RS_TRY(coldots(dt, R, n, R, n, n, np, rrn, st));
        k_cg_update2<T><<<blocks, 256, 0, st>>>(R, P, rr, rrn, n, np);
        k_copy_d<<<1, 64, 0, st>>>(rrn, rr, n);
        RS_LAUNCH_CHECK();
    }
    return RS_OK;
}

int shifted_poisson_cg(rs_ham *h, const void *B, int64_t ldb, void *X, int64_t ldx, int n, int n_iter, int dtype,
                       void *work, cudaStream_t st) {
    if (dtype == RS_F64)
        return cg_t<double>(h, (const double *)B, ldb, (double *)X, ldx, n, n_iter, work, st);
    return cg_t<float>(h, (const float *)B, ldb, (float *)X, ldx, n, n_iter, work, st);
}

// ------------------------------------------------ network on dense tiles ---
// Activations [tile][C][D^3], point index p = (i D + j) D + k.

__device__ __forceinline__ int tap_offset(int t, int D) {
    const int a = t / 9 - 1, b = (t / 3) % 3 - 1, c = t % 3 - 1;
    return (a * D + b) * D + c;
}
__device__ __forceinline__ bool tap_inside(int t, int i, int j, int k, int D) {
    const int a = i + t / 9 - 1, b = j + (t / 3) % 3 - 1, c = k + t % 3 - 1;
    return (unsigned)a < (unsigned)D && (unsigned)b < (unsigned)D && (unsigned)c < (unsigned)D;
}

// z = conv(in), a = relu(z) * mask (or a = z * mask when relu == false)
template <int CIN, int COUT>
__global__ void k_tile_fwd(const float *__restrict__ in, const float *__restrict__ wq, const uint8_t *__restrict__ mask,
                           int ntiles, int D, float *__restrict__ z, float *__restrict__ a, bool relu) {
    __shared__ float w[COUT * CIN * 27];
    for (int e = threadIdx.x; e < COUT * CIN * 27; e += blockDim.x) w[e] = wq[e];
    __syncthreads();
    const int D3 = D * D * D;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)ntiles * D3) return;
    const int tile = (int)(g / D3), p = (int)(g % D3);
    const int i = p / (D * D), j = (p / D) % D, k = p % D;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = 0.f;
    const float *src = in + (int64_t)tile * CIN * D3;
    for (int t = 0; t < 27; ++t) {
        if (!tap_inside(t, i, j, k, D)) continue;
        const int q = p + tap_offset(t, D);
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) {
            const float x = src[(int64_t)ci * D3 + q];
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[co] = fmaf(w[(co * CIN + ci) * 27 + t], x, acc[co]);
        }
    }
    const float m = mask[(int64_t)tile * D3 + p] ? 1.f : 0.f;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        const int64_t o = ((int64_t)tile * COUT + co) * D3 + p;
        if (z) z[o] = acc[co];
        a[o] = (relu ? fmaxf(acc[co], 0.f) : acc[co]) * m;
    }
}

// gin[ci][q] = sum_co sum_t w[co][ci][t] gout[co][q - off_t]
template <int CIN, int COUT>
__global__ void k_tile_bwd_data(const float *__restrict__ gout, const float *__restrict__ wq, int ntiles, int D,
                                float *__restrict__ gin) {
    __shared__ float w[COUT * CIN * 27];
    for (int e = threadIdx.x; e < COUT * CIN * 27; e += blockDim.x) w[e] = wq[e];
    __syncthreads();
    const int D3 = D * D * D;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)ntiles * D3) return;
    const int tile = (int)(g / D3), q = (int)(g % D3);
    const int i = q / (D * D), j = (q / D) % D, k = q % D;
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.f;
    const float *src = gout + (int64_t)tile * COUT * D3;
    for (int t = 0; t < 27; ++t) {
        // output point p = q - off_t exists when the mirrored tap is inside
        if (!tap_inside(26 - t, i, j, k, D)) continue;
        const int p = q - tap_offset(t, D);
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            const float gv = src[(int64_t)co * D3 + p];
#pragma unroll
            for (int ci = 0; ci < CIN; ++ci) acc[ci] = fmaf(w[(co * CIN + ci) * 27 + t], gv, acc[ci]);
        }
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) gin[((int64_t)tile * CIN + ci) * D3 + q] = acc[ci];
}

// dW[co][ci][t] += sum over the tile points p (with p + d_t inside the tile)
// of gout[co][p] * in[ci][p + d_t].  CTA (tile, slab of WB_PLANES planes):
// the slab of gout and the slab plus one plane on either side of `in` are
// staged in shared memory; thread (ci, t) keeps COUT accumulators.
constexpr int WB_PLANES = 2;
template <int CIN, int COUT>
__global__ void k_tile_bwd_weight(const float *__restrict__ gout, const float *__restrict__ in, int ntiles, int D,
                                  float *__restrict__ dW) {
    extern __shared__ float wsm[];
    const int D2 = D * D, D3 = D2 * D;
    const int tile = blockIdx.x, i0 = blockIdx.y * WB_PLANES;
    const int np = min(WB_PLANES, D - i0);
    float *gs = wsm;                               // [COUT][np][D2]
    float *as = wsm + COUT * WB_PLANES * D2;       // [CIN][np + 2][D2], plane i0 - 1 first
    for (int e = threadIdx.x; e < COUT * np * D2; e += blockDim.x) {
        const int co = e / (np * D2), r = e - co * np * D2;
        gs[co * WB_PLANES * D2 + r] = gout[((int64_t)tile * COUT + co) * D3 + (int64_t)i0 * D2 + r];
    }
    for (int e = threadIdx.x; e < CIN * (np + 2) * D2; e += blockDim.x) {
        const int ci = e / ((np + 2) * D2), r = e - ci * (np + 2) * D2;
        const int pl = i0 - 1 + r / D2;
        as[ci * (WB_PLANES + 2) * D2 + r] =
            (pl >= 0 && pl < D) ? in[((int64_t)tile * CIN + ci) * D3 + (int64_t)pl * D2 + r % D2] : 0.f;
    }
    __syncthreads();
    const int w = threadIdx.x;
    if (w >= CIN * 27) return;
    const int ci = w / 27, t = w - ci * 27;
    const int di = t / 9 - 1, dj = (t / 3) % 3 - 1, dk = t % 3 - 1;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = 0.f;
    const float *ab = as + ci * (WB_PLANES + 2) * D2;
    for (int pl = 0; pl < np; ++pl) {
        if ((unsigned)(i0 + pl + di) >= (unsigned)D) continue;   // zero padding outside the tile
        for (int j = max(0, -dj); j < min(D, D - dj); ++j) {
            const float *arow = ab + (pl + 1 + di) * D2 + (j + dj) * D + dk;
            const int gofs = pl * D2 + j * D;
            for (int k = max(0, -dk); k < min(D, D - dk); ++k) {
                const float x = arow[k];
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] = fmaf(gs[co * WB_PLANES * D2 + gofs + k], x, acc[co]);
            }
        }
    }
#pragma unroll
    for (int co = 0; co < COUT; ++co) atomicAdd(dW + (co * CIN + ci) * 27 + t, acc[co]);
}

template <int CIN, int COUT> int tile_bwd_weight(const float *gout, const float *in, int ntiles, int D, float *dW,
                                                 cudaStream_t st) {
    const size_t sm = sizeof(float) * (size_t)(COUT * WB_PLANES + CIN * (WB_PLANES + 2)) * D * D;
    if (sm > 200 * 1024) return fail(RS_EINVAL, "tile_bwd_weight: tile too large");
    RS_TRY(smem_optin((const void *)k_tile_bwd_weight<CIN, COUT>, sm));
    const int threads = ((CIN * 27 + 31) / 32) * 32;
    k_tile_bwd_weight<CIN, COUT><<<dim3((unsigned)ntiles, (unsigned)((D + WB_PLANES - 1) / WB_PLANES)), threads, sm, st>>>(
        gout, in, ntiles, D, dW);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// g = d loss / d y with loss = sum_{valid} (y - t)^2 / nvalid; returns the sum in loss[0]
__global__ void k_tile_loss(const float *__restrict__ y, const float *__restrict__ tgt, const uint8_t *__restrict__ mask,
                            const uint8_t *__restrict__ valid, int ntiles, int D, double inv_n, float *__restrict__ gy,
                            double *loss) {
    __shared__ double red[256];
    const int D3 = D * D * D;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double l = 0.0;
    if (g < (int64_t)ntiles * D3) {
        const int p = (int)(g % D3);
        const bool v = valid[p] && mask[g];
        const float d = v ? y[g] - tgt[g] : 0.f;
        gy[g] = (float)(2.0 * inv_n) * d;
        l = (double)d * d * inv_n;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// g *= mask * (z > 0) (relu derivative; the mask is folded in)
__global__ void k_relu_grad(float *g, const float *z, const uint8_t *mask, int ntiles, int C, int D) {
    const int D3 = D * D * D;
    const int64_t n = (int64_t)ntiles * C * D3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = e / ((int64_t)C * D3);
        const int p = (int)(e % D3);
        if (!(mask[tile * D3 + p] && z[e] > 0.f)) g[e] = 0.f;
    }
}

__global__ void k_mask_grad(float *g, const uint8_t *mask, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        if (!mask[e]) g[e] = 0.f;
}

__global__ void k_round_weights(const float *w, float *wq, int n) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) wq[e] = bf16_round(w[e]);
}

__global__ void k_round_inputs(const float *x, float *xq, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        xq[e] = bf16_round(x[e]);
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       int step) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float mh = mm / (1.f - powf(b1, (float)step));
    const float vh = vv / (1.f - powf(b2, (float)step));
    w[e] -= lr * mh / (sqrtf(vh) + eps);
}

// Network forward + backward on a batch of dense tiles; activations in `ws`.
struct TileBufs {
    float *x0, *z1, *a1, *z2, *a2, *y, *g3, *ga2, *ga1, *wq;
    static size_t floats(int ntiles, int D) {
        const size_t v = (size_t)ntiles * D * D * D;
        return v * (1 + NC * 4 + 1 + 1 + NC * 2) + W_TOTAL + 64;
    }
    TileBufs(float *base, int ntiles, int D) {
        const size_t v = (size_t)ntiles * D * D * D;
        x0 = base;
        z1 = x0 + v;
        a1 = z1 + NC * v;
        z2 = a1 + NC * v;
        a2 = z2 + NC * v;
        y = a2 + NC * v;
        g3 = y + v;
        ga2 = g3 + v;
        ga1 = ga2 + NC * v;
        wq = ga1 + NC * v;
    }
};

int tile_forward(const float *wq, const float *x0, const uint8_t *mask, int ntiles, int D, TileBufs &b, cudaStream_t st) {
    const int64_t n = (int64_t)ntiles * D * D * D;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    k_tile_fwd<1, NC><<<blocks, 128, 0, st>>>(x0, wq + W1_OFF, mask, ntiles, D, b.z1, b.a1, true);
    k_tile_fwd<NC, NC><<<blocks, 128, 0, st>>>(b.a1, wq + W2_OFF, mask, ntiles, D, b.z2, b.a2, true);
    k_tile_fwd<NC, 1><<<blocks, 128, 0, st>>>(b.a2, wq + W3_OFF, mask, ntiles, D, nullptr, b.y, false);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// grad (2160 floats) must be zeroed by the caller; g3 holds d loss / d y.
int tile_backward(const float *wq, const float *x0, const uint8_t *mask, int ntiles, int D, TileBufs &b, float *grad,
                  cudaStream_t st) {
    const int64_t n = (int64_t)ntiles * D * D * D;
    const unsigned blocks = (unsigned)((n + 127) / 128);

    k_mask_grad<<<1024, 256, 0, st>>>(b.g3, mask, n);
    RS_TRY((tile_bwd_weight<NC, 1>(b.g3, b.a2, ntiles, D, grad + W3_OFF, st)));
    k_tile_bwd_data<NC, 1><<<blocks, 128, 0, st>>>(b.g3, wq + W3_OFF, ntiles, D, b.ga2);
    k_relu_grad<<<1024, 256, 0, st>>>(b.ga2, b.z2, mask, ntiles, NC, D);
    RS_TRY((tile_bwd_weight<NC, NC>(b.ga2, b.a1, ntiles, D, grad + W2_OFF, st)));
    k_tile_bwd_data<NC, NC><<<blocks, 128, 0, st>>>(b.ga2, wq + W2_OFF, ntiles, D, b.ga1);
    k_relu_grad<<<1024, 256, 0, st>>>(b.ga1, b.z1, mask, ntiles, NC, D);
    RS_TRY((tile_bwd_weight<1, NC>(b.ga1, x0, ntiles, D, grad + W1_OFF, st)));
    RS_LAUNCH_CHECK();
    return RS_OK;
}

// ------------------------------------------------------ tile extraction ---
// For tile n: column col[n], interior origin (bbox-local) o[n] (a 16^3 box
// starting 3 points inside the D^3 tile).  x = r / rms, t = xcg / rms,
// mask = grid membership.
__global__ void k_cut_tiles(const int32_t *__restrict__ map, int d0, int d1, int d2, const float *__restrict__ R,
                            const float *__restrict__ X, int64_t ld, const double *__restrict__ rms,
                            const int4 *__restrict__ org, int ntiles, int D, float *__restrict__ xin,
                            float *__restrict__ tgt, uint8_t *__restrict__ mask) {
    const int D3 = D * D * D;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)ntiles * D3) return;
    const int n = (int)(g / D3), p = (int)(g % D3);
    const int4 o = org[n];
    const int a = o.y + p / (D * D), b = o.z + (p / D) % D, c = o.w + p % D;
    int r = -1;
    if ((unsigned)a < (unsigned)d0 && (unsigned)b < (unsigned)d1 && (unsigned)c < (unsigned)d2)
        r = map[((int64_t)a * d1 + b) * d2 + c];
    const float s = (float)(1.0 / rms[o.x]);
    xin[g] = r >= 0 ? bf16_round(R[(int64_t)r * ld + o.x] * s) : 0.f;
    tgt[g] = r >= 0 ? X[(int64_t)r * ld + o.x] * s : 0.f;
    mask[g] = r >= 0;
}

__global__ void k_rms(const double *ss, int n, double inv_np, double *rms) {
    const int k = threadIdx.x;
    if (k < n) rms[k] = ss[k] > 0 ? sqrt(ss[k] * inv_np) : 1.0;
}

// --------------------------------------------- inference on the grid ---

// xhat = bf16(r / rms) and the per-column rms
__global__ void k_net_input(const float *__restrict__ R, int64_t ldr, const double *__restrict__ rms, int nb,
                            int npts, float *__restrict__ x) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts * nb) return;
    const int p = t / nb, s = t - p * nb;
    x[t] = bf16_round(R[(int64_t)p * ldr + s] * (float)(1.0 / rms[s]));
}

// layer on the grid: out[p][co][s] = act(sum_t sum_ci w[co][ci][t] in[nbr_t(p)][ci][s]).
// The layer's weights (BF16 values) are staged in shared memory as
// [tap][ci][co], so one 16-byte load gives four output channels' weights
// (a broadcast: every lane reads the same word).
template <int CIN, int COUT, bool RELU, bool FINAL, int WOFF>
__global__ void __launch_bounds__(256) k_net_layer(const int32_t *__restrict__ map, const int32_t *__restrict__ loc,
                                                   int d1, int d2, int npts, int nb, const float *__restrict__ wq,
                                                   const float *__restrict__ in, float *__restrict__ out, int64_t ldo,
                                                   const double *__restrict__ rms) {
    constexpr int CO4 = (COUT + 3) / 4 * 4;
    __shared__ __align__(16) float ws[27 * CIN * CO4];
    for (int e = threadIdx.x; e < 27 * CIN * CO4; e += blockDim.x) {
        const int co = e % CO4, ci = (e / CO4) % CIN, tap = e / (CO4 * CIN);
        ws[e] = co < COUT ? __ldg(wq + WOFF + (co * CIN + ci) * 27 + tap) : 0.f;
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts * nb) return;
    const int p = t / nb, s = t - p * nb;
    const int64_t L = __ldg(loc + p);
    float acc[CO4];
#pragma unroll
    for (int co = 0; co < CO4; ++co) acc[co] = 0.f;
#pragma unroll 3
    for (int tap = 0; tap < 27; ++tap) {
        const int64_t off = ((int64_t)(tap / 9 - 1) * d1 + ((tap / 3) % 3 - 1)) * d2 + (tap % 3 - 1);
        const int q = __ldg(map + L + off);
        if (q < 0) continue;
        const float *src = in + ((int64_t)q * CIN) * nb + s;
        const float4 *w4 = reinterpret_cast<const float4 *>(ws + tap * CIN * CO4);
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) {
            const float x = __ldg(src + (int64_t)ci * nb);
#pragma unroll
            for (int c4 = 0; c4 < CO4 / 4; ++c4) {
                const float4 w = w4[ci * (CO4 / 4) + c4];
                acc[4 * c4 + 0] = fmaf(w.x, x, acc[4 * c4 + 0]);
                if (4 * c4 + 1 < COUT) acc[4 * c4 + 1] = fmaf(w.y, x, acc[4 * c4 + 1]);
                if (4 * c4 + 2 < COUT) acc[4 * c4 + 2] = fmaf(w.z, x, acc[4 * c4 + 2]);
                if (4 * c4 + 3 < COUT) acc[4 * c4 + 3] = fmaf(w.w, x, acc[4 * c4 + 3]);
            }
        }
    }
    if (FINAL) {
        out[(int64_t)p * ldo + s] = acc[0] * (float)rms[s];
    } else {
#pragma unroll
        for (int co = 0; co < COUT; ++co) out[((int64_t)p * COUT + co) * nb + s] = RELU ? fmaxf(acc[co], 0.f) : acc[co];
    }
}

}  // namespace rs

using namespace rs;

// ---------------------------------------------------------------- C ABI ---

extern "C" int64_t rs_cg_workspace_bytes(int64_t npts, int ncols, int dtype) {
    if (npts < 1 || ncols < 1 || ncols > 64) return -1;
    return cg_workspace_bytes(npts, ncols, dtype);
}

extern "C" int rs_shifted_poisson_cg(rs_ham *h, const void *B_dev, void *X_dev, int64_t ld, int ncols, int n_iter,
                                     int dtype, void *work_dev, void *stream) {
    if (!h || !B_dev || !X_dev || !work_dev) return fail(RS_EINVAL, "rs_shifted_poisson_cg: null argument");
    if (ncols < 1 || ncols > 64 || (ncols & (ncols - 1))) return fail(RS_EINVAL, "rs_shifted_poisson_cg: ncols must be a power of two <= 64");
    if (ld < ncols || n_iter < 0) return fail(RS_EINVAL, "rs_shifted_poisson_cg: bad ld or n_iter");
    if (dtype != RS_F64 && dtype != RS_F32) return fail(RS_EINVAL, "rs_shifted_poisson_cg: bad dtype");
    return shifted_poisson_cg(h, B_dev, ld, X_dev, ld, ncols, n_iter, dtype, work_dev, (cudaStream_t)stream);
}

extern "C" int rs_convnet_tiles(const float *w_dev, const float *x_dev, const uint8_t *mask_dev, const float *target_dev,
                                const uint8_t *valid_dev, int ntiles, int D, float *y_dev, float *grad_dev,
                                double *loss_host, void *stream) {
    if (!w_dev || !x_dev || !mask_dev || !y_dev || ntiles < 1 || D < 3)
        return fail(RS_EINVAL, "rs_convnet_tiles: bad arguments");
    if ((grad_dev || loss_host) && (!target_dev || !valid_dev))
        return fail(RS_EINVAL, "rs_convnet_tiles: gradients need target and valid");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf ws, dl;
    RS_TRY(ws.alloc(TileBufs::floats(ntiles, D) * sizeof(float)));
    RS_TRY(dl.alloc(sizeof(double)));
    TileBufs b(ws.as<float>(), ntiles, D);
    const int64_t n = (int64_t)ntiles * D * D * D;
    k_round_weights<<<9, 256, 0, st>>>(w_dev, b.wq, W_TOTAL);
    k_round_inputs<<<1024, 256, 0, st>>>(x_dev, b.x0, n);
    RS_LAUNCH_CHECK();
    RS_TRY(tile_forward(b.wq, b.x0, mask_dev, ntiles, D, b, st));
    RS_CUDA(cudaMemcpyAsync(y_dev, b.y, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    if (grad_dev || loss_host) {
        int nvalid = 0;
        {
            std::vector<uint8_t> v((size_t)D * D * D), m((size_t)n);
            RS_CUDA(cudaMemcpyAsync(v.data(), valid_dev, v.size(), cudaMemcpyDeviceToHost, st));
            RS_CUDA(cudaMemcpyAsync(m.data(), mask_dev, m.size(), cudaMemcpyDeviceToHost, st));
            RS_CUDA(cudaStreamSynchronize(st));
            const int D3 = D * D * D;
            for (int64_t e = 0; e < n; ++e) nvalid += (v[e % D3] && m[e]);
        }
        RS_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), st));
        k_tile_loss<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b.y, target_dev, mask_dev, valid_dev, ntiles, D,
                                                                1.0 / std::max(nvalid, 1), b.g3, dl.as<double>());
        RS_LAUNCH_CHECK();
        if (grad_dev) {
            RS_CUDA(cudaMemsetAsync(grad_dev, 0, sizeof(float) * W_TOTAL, st));
            RS_TRY(tile_backward(b.wq, b.x0, mask_dev, ntiles, D, b, grad_dev, st));
        }
        if (loss_host) RS_CUDA(cudaMemcpyAsync(loss_host, dl.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

// splitmix64: the seeded generator of the tile positions
static uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

namespace rs {

// Adam on dense tiles already cut: `epochs` passes over the tiles in order,
// one step per batch of `batch` consecutive tiles (a last partial batch is
// dropped), moments zero at the start.  loss_host[ep] (may be NULL) gets the
// mean batch loss of epoch ep.  Blocking.
int train_tiles_impl(float *w_dev, const float *xin, const float *tgt, const uint8_t *msk, const uint8_t *dvalid,
                     int ntiles, int D, int batch, int epochs, float lr, float *loss_host, cudaStream_t st) {
    const int D3 = D * D * D;
    const int64_t ntot = (int64_t)ntiles * D3;
    const int B = std::min(batch, ntiles);
    DevBuf ws, grad, m, v, dl;
    RS_TRY(ws.alloc(TileBufs::floats(B, D) * sizeof(float)));
    RS_TRY(grad.alloc(sizeof(float) * W_TOTAL));
    RS_TRY(m.alloc(sizeof(float) * W_TOTAL));
    RS_TRY(v.alloc(sizeof(float) * W_TOTAL));
    RS_TRY(dl.alloc(sizeof(double)));
    RS_CUDA(cudaMemsetAsync(m.p, 0, sizeof(float) * W_TOTAL, st));
    RS_CUDA(cudaMemsetAsync(v.p, 0, sizeof(float) * W_TOTAL, st));
    // number of valid points (interior grid points) of every tile, for the mean
    std::vector<int> tvalid((size_t)ntiles, 0);
    {
        std::vector<uint8_t> hm((size_t)ntot), valid((size_t)D3);
        RS_CUDA(cudaMemcpyAsync(hm.data(), msk, hm.size(), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaMemcpyAsync(valid.data(), dvalid, valid.size(), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
        std::vector<int> vidx;
        for (int e = 0; e < D3; ++e)
            if (valid[e]) vidx.push_back(e);
        for (int n = 0; n < ntiles; ++n) {
            const uint8_t *tm = hm.data() + (size_t)n * D3;
            int cnt = 0;
            for (int e : vidx) cnt += tm[e] != 0;
            tvalid[n] = cnt;
        }
    }
    TileBufs b(ws.as<float>(), B, D);
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        RS_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), st));
        int nbatches = 0;
        for (int t0 = 0; t0 + B <= ntiles; t0 += B, ++nbatches) {
            int nvalid = 0;
            for (int n = t0; n < t0 + B; ++n) nvalid += tvalid[n];
            const float *x0 = xin + (int64_t)t0 * D3;
            const uint8_t *mk = msk + (int64_t)t0 * D3;
            k_round_weights<<<9, 256, 0, st>>>(w_dev, b.wq, W_TOTAL);
            RS_LAUNCH_CHECK();
            RS_TRY(tile_forward(b.wq, x0, mk, B, D, b, st));
            const int64_t n = (int64_t)B * D3;
            k_tile_loss<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b.y, tgt + (int64_t)t0 * D3, mk, dvalid, B, D,
                                                                    1.0 / std::max(nvalid, 1), b.g3, dl.as<double>());
            RS_CUDA(cudaMemsetAsync(grad.p, 0, sizeof(float) * W_TOTAL, st));
            RS_TRY(tile_backward(b.wq, x0, mk, B, D, b, grad.as<float>(), st));
            ++step;
            k_adam<<<(W_TOTAL + 255) / 256, 256, 0, st>>>(w_dev, grad.as<float>(), m.as<float>(), v.as<float>(), W_TOTAL,
                                                          lr, 0.9f, 0.999f, 1e-8f, step);
            RS_LAUNCH_CHECK();
        }
        double tot = 0;
        RS_CUDA(cudaMemcpyAsync(&tot, dl.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
        if (loss_host) loss_host[ep] = (float)(tot / std::max(nbatches, 1));
    }
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

// Cuts c.n_tiles tiles around random grid points of the column pairs (R, X),
// inputs and targets scaled by the residual column's rms, and trains on them.
int train_pairs_impl(const rs_ham *h, const rs_grid *g, const float *R_dev, const float *X_dev, int64_t ld, int ncols,
                     const rs_train_cfg &c, float *w_dev, float *loss_host, cudaStream_t st) {
    const int D = c.tile + 6, D3 = D * D * D;
    const int64_t np = g->npts;
    // tile positions: a random grid point of a random column at the tile centre
    std::vector<int4> org((size_t)c.n_tiles);
    uint64_t seed = c.seed;
    for (int n = 0; n < c.n_tiles; ++n) {
        const int col = (int)(splitmix64(seed) % (uint64_t)ncols);
        const int64_t p = (int64_t)(splitmix64(seed) % (uint64_t)np);
        const int a = g->ijk[3 * p] - g->origin[0], b = g->ijk[3 * p + 1] - g->origin[1], cc = g->ijk[3 * p + 2] - g->origin[2];
        org[n] = make_int4(col, a - D / 2, b - D / 2, cc - D / 2);
    }
    std::vector<uint8_t> valid((size_t)D3, 0);
    for (int i = 3; i < D - 3; ++i)
        for (int j = 3; j < D - 3; ++j)
            for (int k = 3; k < D - 3; ++k) valid[((size_t)i * D + j) * D + k] = 1;
    DevBuf dorg, dvalid, xin, tgt, msk, ss, rms;
    RS_TRY(dorg.upload(org.data(), org.size() * sizeof(int4)));
    RS_TRY(dvalid.upload(valid.data(), valid.size()));
    RS_TRY(xin.alloc((size_t)c.n_tiles * D3 * sizeof(float)));
    RS_TRY(tgt.alloc((size_t)c.n_tiles * D3 * sizeof(float)));
    RS_TRY(msk.alloc((size_t)c.n_tiles * D3));
    RS_TRY(ss.alloc(sizeof(double) * 256));
    RS_TRY(rms.alloc(sizeof(double) * 256));
    RS_TRY(coldots(RS_F32, R_dev, ld, R_dev, ld, ncols, np, ss.as<double>(), st));
    k_rms<<<1, 256, 0, st>>>(ss.as<double>(), ncols, 1.0 / (double)np, rms.as<double>());
    RS_LAUNCH_CHECK();
    const int64_t ntot = (int64_t)c.n_tiles * D3;
    k_cut_tiles<<<(unsigned)((ntot + 255) / 256), 256, 0, st>>>(
        ham_map(h), g->dims[0], g->dims[1], g->dims[2], R_dev, X_dev, ld, rms.as<double>(), dorg.as<int4>(), c.n_tiles,
        D, xin.as<float>(), tgt.as<float>(), msk.as<uint8_t>());
    RS_LAUNCH_CHECK();
    return train_tiles_impl(w_dev, xin.as<float>(), tgt.as<float>(), msk.as<uint8_t>(), dvalid.as<uint8_t>(), c.n_tiles,
                            D, c.batch, c.epochs, c.lr, loss_host, st);
}

}  // namespace rs

extern "C" int rs_precond_train_pairs(rs_ham *h, const rs_grid *g, const float *R_dev, const float *X_dev, int64_t ld,
                                      int ncols, const rs_train_cfg *cfg, float *w_dev, float *loss_host, void *stream) {
    if (!h || !g || !R_dev || !X_dev || !cfg || !w_dev) return fail(RS_EINVAL, "rs_precond_train_pairs: null argument");
    const rs_train_cfg c = *cfg;
    if (ncols < 1 || ncols > 256 || ld < ncols || c.n_tiles < 1 || c.batch < 1 || c.epochs < 0 || c.tile < 1)
        return fail(RS_EINVAL, "rs_precond_train_pairs: bad sizes");
    if (ham_npts(h) != g->npts) return fail(RS_EINVAL, "rs_precond_train_pairs: grid and Hamiltonian differ");
    return train_pairs_impl(h, g, R_dev, X_dev, ld, ncols, c, w_dev, loss_host, (cudaStream_t)stream);
}

extern "C" int rs_precond_train_tiles(float *w_dev, const float *x_dev, const uint8_t *mask_dev, const float *target_dev,
                                      const uint8_t *valid_dev, int ntiles, int D, int batch, int epochs, float lr,
                                      float *loss_host, void *stream) {
    if (!w_dev || !x_dev || !mask_dev || !target_dev || !valid_dev) return fail(RS_EINVAL, "rs_precond_train_tiles: null argument");
    if (ntiles < 1 || D < 3 || D > 64 || batch < 1 || epochs < 0 || !(lr > 0))
        return fail(RS_EINVAL, "rs_precond_train_tiles: bad sizes");
    return train_tiles_impl(w_dev, x_dev, target_dev, mask_dev, valid_dev, ntiles, D, batch, epochs, lr, loss_host,
                            (cudaStream_t)stream);
}

// ----------------------------------------------------- solver plug-in ---

namespace rs {

int learned_apply(const rs_ham *h, const float *R, int64_t ldr, float *W, int64_t ldw, int nb, const float *wq_dev,
                  float *act, double *dots, cudaStream_t st) {
    const int64_t np = ham_npts(h);
    double *ss = dots, *rms = dots + 64;
    RS_TRY(coldots(RS_F32, R, ldr, R, ldr, nb, np, ss, st));
    k_rms<<<1, 64, 0, st>>>(ss, nb, 1.0 / (double)np, rms);
    if (np * nb >= (int64_t)INT32_MAX) return fail(RS_EINVAL, "learned preconditioner: npts * nb above 2^31");
    const int n32 = (int)np;
    float *x = act, *a1 = x + np * nb, *a2 = a1 + np * NC * nb;
    const unsigned blocks = (unsigned)((np * nb + 255) / 256);
    k_net_input<<<blocks, 256, 0, st>>>(R, ldr, rms, nb, n32, x);
    const int32_t *map = ham_map(h), *loc = ham_loc(h);
    const int d1 = ham_dim(h, 1), d2 = ham_dim(h, 2);
    k_net_layer<1, NC, true, false, W1_OFF><<<blocks, 256, 0, st>>>(map, loc, d1, d2, n32, nb, wq_dev, x, a1, 0, rms);
    k_net_layer<NC, NC, true, false, W2_OFF><<<blocks, 256, 0, st>>>(map, loc, d1, d2, n32, nb, wq_dev, a1, a2, 0, rms);
    k_net_layer<NC, 1, false, true, W3_OFF><<<blocks, 256, 0, st>>>(map, loc, d1, d2, n32, nb, wq_dev, a2, W, ldw, rms);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

int64_t learned_act_floats(int64_t npts, int nb) { return npts * nb * (1 + 2 * NC); }

int learned_round_weights(const float *w, float *wq, cudaStream_t st) {
    k_round_weights<<<9, 256, 0, st>>>(w, wq, W_TOTAL);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

}  // namespace rs

extern "C" int rs_precond_apply(rs_ham *h, const float *w_dev, const float *R_dev, int64_t ldr, float *W_dev, int64_t ldw,
                                int nb, void *stream) {
    if (!h || !w_dev || !R_dev || !W_dev) return fail(RS_EINVAL, "rs_precond_apply: null argument");
    if (nb < 1 || nb > 64 || ldr < nb || ldw < nb) return fail(RS_EINVAL, "rs_precond_apply: bad nb or ld");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf *ws = ham_scratch(h, (sizeof(float) * (size_t)(LEARNED_WEIGHTS + learned_act_floats(ham_npts(h), nb))) +
                                    sizeof(double) * 128);
    if (!ws) return fail(RS_ENOMEM, "rs_precond_apply: device allocation failed");
    double *dots = ws->as<double>();
    float *wq = reinterpret_cast<float *>(dots + 128);
    float *act = wq + LEARNED_WEIGHTS;
    RS_TRY(learned_round_weights(w_dev, wq, st));
    return learned_apply(h, R_dev, ldr, W_dev, ldw, nb, wq, act, dots, st);
}

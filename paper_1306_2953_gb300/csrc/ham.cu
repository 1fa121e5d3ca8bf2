// Kohn-Sham Hamiltonian applied to a block of orbitals (Sec. V, Eq. 3).
//
// Two launches per block:
//  1. k_project: the Kleinman-Bylander projection integrals of Eq. (4),
//     c[A,q,s] = E[A,q] dV sum_{p in S_A} gamma_Aq(p) psi(p,s), PSPLIT CTAs
//     per (atom, state group), each a block-wide tree reduction over its share
//     of the sphere points added to the zeroed coefficients; stored
//     [atom][state][q] so that one 16-byte load gives a state's four.
//  2. k_stencil: the 25-point star kinetic stencil (Sec. V.A), the local
//     potential (Sec. V.B) and the nonlocal sum of Eq. (4), fused.  Each CTA
//     owns a TX x TY column of lattice points (axes 2 and 1 of the point
//     map) and one group of SG states, and marches along axis 0.  Every
//     thread keeps a 2x2 patch of columns for one state in registers with a
//     9-deep queue along the march axis, so the axis-0 neighbours come from
//     registers; the current plane (interior written from the queues, the
//     4-point x/y halos staged by cp.async three planes deep) sits in shared
//     memory for the axis-1/axis-2 neighbours.  The nonlocal term is a
//     gather: each output point sums over the atoms whose spheres cover it,
//     so overlapping spheres need neither atom colouring (Sec. V.C, Fig. 10)
//     nor atomics, and the output is written exactly once.
// Orbitals are [npts][ld] with the state index fastest (Sec. IV, Fig. 4b);
// grid points are addressed through the int32 point map (Sec. V.A).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "device.h"
#include "ham.h"
#include "stencil_ring.h"

#ifndef RS_STENCIL_V3
#define RS_STENCIL_V3 0
#endif

// 1: FP32 blocks of 32 states go to the persistent ring-buffer kernel
// (stencil_ring.cu) when the block's layout allows 16-byte row copies.
#ifndef RS_STENCIL_RING
#define RS_STENCIL_RING 1
#endif

// Height (planes) of the z-slabs of that kernel's work units.
#ifndef RS_RING_SLAB
#define RS_RING_SLAB 32
#endif

#ifndef RS_STENCIL_MINB_F32
#define RS_STENCIL_MINB_F32 1
#endif

namespace rs {

template <typename T> struct HamDev {
    const int4 *pinfo;  // per point: nonlocal entry range [x, y) and V (z: float bits; z,w: double bits)
    const int32_t *map;
    int d0, d1, d2;
    const T *V;
    const int32_t *cov_off, *cov_atom;
    const T *cov_gam;   // [entries][4]
    const int32_t *sph_off, *sph_idx;
    const T *sph_gam;   // [entries][4]
    const T *E;         // [atoms][4]
    T dV;
    T w[5];             // w[0] = 3 kin c_0, w[j] = kin c_j, kin = -1/(2h^2)
};

// ---------------------------------------------------------------- helpers --

template <typename T> __device__ __forceinline__ T point_v(int4 inf);
template <> __device__ __forceinline__ float point_v<float>(int4 inf) { return __int_as_float(inf.z); }
template <> __device__ __forceinline__ double point_v<double>(int4 inf) { return __hiloint2double(inf.w, inf.z); }

template <int BYTES> __device__ __forceinline__ void cp_async(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int sz = valid ? BYTES : 0;
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES), "r"(sz)
                     : "memory");
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T> struct Four { T a, b, c, d; };
__device__ __forceinline__ Four<float> load4(const float *p) {
    float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Four<double> load4(const double *p) {
    double2 u = __ldg(reinterpret_cast<const double2 *>(p));
    double2 v = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return {u.x, u.y, v.x, v.y};
}

// ------------------------------------------------- projection integrals ---

// Grid (atoms * PSPLIT, state groups): each CTA sums 1/PSPLIT of an atom's
// sphere points and adds its partial sums to the (zeroed) coefficients.
constexpr int PSPLIT = 8;

template <typename T, int SGP, int NT>
__global__ void __launch_bounds__(NT) k_project(HamDev<T> d, const T *__restrict__ psi, int64_t ldp, int nb,
                                                T *__restrict__ cproj) {
    constexpr int R = NT / SGP;
    __shared__ T red[4][NT];
    const int A = blockIdx.x / PSPLIT, part = blockIdx.x % PSPLIT;
    const int sg0 = blockIdx.y * SGP;
    const int s = threadIdx.x % SGP, r = threadIdx.x / SGP;
    const int o = __ldg(d.sph_off + A), e = __ldg(d.sph_off + A + 1);
    const int len = e - o, per = (len + PSPLIT - 1) / PSPLIT;
    const int i0 = o + part * per, i1 = min(e, i0 + per);
    const T *ps = psi + sg0 + s;
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 8
    for (int i = i0 + r; i < i1; i += R) {
        const int p = __ldg(d.sph_idx + i);
        const T v = __ldg(ps + (int64_t)p * ldp);
        const Four<T> g = load4(d.sph_gam + 4 * (int64_t)i);
        a0 += g.a * v;
        a1 += g.b * v;
        a2 += g.c * v;
        a3 += g.d * v;
    }
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    red[3][threadIdx.x] = a3;
    __syncthreads();
    for (int st = R / 2; st > 0; st >>= 1) {
        if (r < st) {
#pragma unroll
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st * SGP];
        }
        __syncthreads();
    }
    if (r == 0 && i0 < i1) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            atomicAdd(cproj + ((int64_t)A * nb + sg0 + s) * 4 + q, __ldg(d.E + 4 * A + q) * d.dV * red[q][s]);
    }
}

// ------------------------------------------- fused stencil + V + nonlocal ---

// Maximum number of planes of one work item (the z chunk).
constexpr int ZCHUNK = 32;

template <typename T, int SG, int TX, int TY> struct StencilCfg {
    static constexpr int W2 = TX + 8, W1 = TY + 8;
    static constexpr int PLANE = W1 * W2 * SG;
    static constexpr int NT = (TX / 2) * (TY / 2) * SG;
    static constexpr int RING = 3;
    static constexpr int CHB = (SG * (int)sizeof(T) >= 16) ? 16 : SG * (int)sizeof(T);
    static constexpr int CHE = CHB / (int)sizeof(T);
    static constexpr int CPR = SG / CHE;
    static constexpr int NH = 8 * TY + 8 * TX;
    static constexpr int HPT = (NH * CPR + NT - 1) / NT;     // halo copies per thread and plane
    static constexpr int NI = TX * TY;
    static constexpr bool STAGE = NI <= 128;                  // stage interior rows in shared memory
    static constexpr int NROW = STAGE ? (ZCHUNK + 9) * NI : 0;
    static constexpr size_t SMEM = (size_t)RING * PLANE * sizeof(T) + (size_t)NROW * sizeof(int);
    static constexpr int MINB = sizeof(T) == 4 ? RS_STENCIL_MINB_F32 : 1;
};

template <typename T, int SG, int TX, int TY>
__global__ void __launch_bounds__(StencilCfg<T, SG, TX, TY>::NT, StencilCfg<T, SG, TX, TY>::MINB)
    k_stencil(HamDev<T> d, const T *__restrict__ psi, int64_t ldp, T *__restrict__ hpsi, int64_t ldh,
              const T *__restrict__ cproj, int nb, const int4 *__restrict__ work) {
    using C = StencilCfg<T, SG, TX, TY>;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    int *rows = reinterpret_cast<int *>(smraw + (size_t)C::RING * C::PLANE * sizeof(T));

    const int tid = threadIdx.x;
    const int s = tid % SG;
    const int patch = tid / SG;
    const int lx = 2 * (patch % (TX / 2));
    const int ly = 2 * (patch / (TX / 2));
    const int4 wk = work[blockIdx.x];
    const int b1 = wk.x * TY, b2 = wk.y * TX;
    const int za = wk.z, zb = wk.w;
    const int sg0 = blockIdx.y * SG;
    const T *psig = psi + sg0;

    auto map_at = [&](int a0, int a1, int a2) -> int {
        if ((unsigned)a0 >= (unsigned)d.d0 || (unsigned)a1 >= (unsigned)d.d1 || (unsigned)a2 >= (unsigned)d.d2)
            return -1;
        return __ldg(d.map + ((int64_t)a0 * d.d1 + a1) * d.d2 + a2);
    };
    // interior point rows of planes za-4 .. zb+4, staged once per work item
    if constexpr (C::STAGE) {
        const int nrow = (zb - za + 9) * C::NI;
        for (int e = tid; e < nrow; e += C::NT) {
            const int pl = e / C::NI, pos = e % C::NI;
            rows[e] = map_at(za - 4 + pl, b1 + pos / TX, b2 + pos % TX);
        }
    }
    auto row_of = [&](int z, int iy, int ix) -> int {
        if constexpr (C::STAGE) return rows[(z - za + 4) * C::NI + iy * TX + ix];
        return map_at(z, b1 + iy, b2 + ix);
    };
    auto load_val = [&](int r) -> T { return r >= 0 ? __ldg(psig + (int64_t)r * ldp + s) : T(0); };

    // this thread's halo copies j < HPT: copy index i = tid + j NT -> (hy, hx, chunk)
    auto halo_pos = [&](int i, int &hy, int &hx, int &c) {
        const int hh = i / C::CPR;
        c = i % C::CPR;
        if (hh < 8 * TY) {
            hy = hh >> 3;
            const int t = hh & 7;
            hx = t < 4 ? t - 4 : TX + t - 4;
        } else {
            const int h2 = hh - 8 * TY;
            hx = h2 % TX;
            const int t = h2 / TX;
            hy = t < 4 ? t - 4 : TY + t - 4;
        }
    };
    int hr[C::HPT];
    auto halo_rows = [&](int z) {
#pragma unroll
        for (int j = 0; j < C::HPT; ++j) {
            const int i = tid + j * C::NT;
            int hy, hx, c;
            halo_pos(i, hy, hx, c);
            hr[j] = i < C::NH * C::CPR ? map_at(z, b1 + hy, b2 + hx) : -1;
        }
    };
    auto issue_halo = [&](int slot) {
        T *base = sm + slot * C::PLANE;
#pragma unroll
        for (int j = 0; j < C::HPT; ++j) {
            const int i = tid + j * C::NT;
            if (i >= C::NH * C::CPR) continue;
            int hy, hx, c;
            halo_pos(i, hy, hx, c);
            const T *src = hr[j] >= 0 ? psig + (int64_t)hr[j] * ldp + c * C::CHE : psig;
            cp_async<C::CHB>(base + ((hy + 4) * C::W2 + (hx + 4)) * SG + c * C::CHE, src, hr[j] >= 0);
        }
    };
    __syncthreads();

    T q[2][2][9];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) q[dy][dx][k] = load_val(row_of(za - 4 + k, ly + dy, lx + dx));

    halo_rows(za);
    issue_halo(0);
    cp_async_commit();
    halo_rows(za + 1);
    if (za + 1 < zb) issue_halo(1);
    cp_async_commit();
    halo_rows(za + 2);

    const T w0 = d.w[0], w1 = d.w[1], w2 = d.w[2], w3 = d.w[3], w4 = d.w[4];
    int slot = 0;
    for (int z = za; z < zb; ++z) {
        const int pslot = slot == 0 ? 2 : slot - 1;  // (slot + 2) % 3
        if (z + 2 < zb) issue_halo(pslot);
        cp_async_commit();

        T nq[2][2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) nq[dy][dx] = load_val(row_of(z + 5, ly + dy, lx + dx));

        T *P = sm + slot * C::PLANE;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) P[((ly + dy + 4) * C::W2 + lx + dx + 4) * SG + s] = q[dy][dx][4];
        cp_async_wait<2>();
        __syncthreads();

        // axis-0 neighbours from the register queues
        T acc[2][2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                acc[dy][dx] = w0 * q[dy][dx][4] + w1 * (q[dy][dx][5] + q[dy][dx][3]) +
                              w2 * (q[dy][dx][6] + q[dy][dx][2]) + w3 * (q[dy][dx][7] + q[dy][dx][1]) +
                              w4 * (q[dy][dx][8] + q[dy][dx][0]);
            }
        // axis-2 neighbours: one row of 10 values per patch row (8 from shared memory)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            T v[10];
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (k != 4 && k != 5) v[k] = P[((ly + dy + 4) * C::W2 + lx + k) * SG + s];
            v[4] = q[dy][0][4];
            v[5] = q[dy][1][4];
#pragma unroll
            for (int dx = 0; dx < 2; ++dx)
                acc[dy][dx] += w1 * (v[5 + dx] + v[3 + dx]) + w2 * (v[6 + dx] + v[2 + dx]) +
                               w3 * (v[7 + dx] + v[1 + dx]) + w4 * (v[8 + dx] + v[0 + dx]);
        }
        // axis-1 neighbours: one column of 10 values per patch column
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            T v[10];
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (k != 4 && k != 5) v[k] = P[((ly + k) * C::W2 + lx + dx + 4) * SG + s];
            v[4] = q[0][dx][4];
            v[5] = q[1][dx][4];
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
                acc[dy][dx] += w1 * (v[5 + dy] + v[3 + dy]) + w2 * (v[6 + dy] + v[2 + dy]) +
                               w3 * (v[7 + dy] + v[1 + dy]) + w4 * (v[8 + dy] + v[0 + dy]);
        }
        // local potential, nonlocal gather, store
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int r = row_of(z, ly + dy, lx + dx);
                if (r < 0) continue;
                const int4 inf = __ldg(d.pinfo + r);
                T out = acc[dy][dx] + point_v<T>(inf) * q[dy][dx][4];
                for (int e = inf.x; e < inf.y; ++e) {
                    const int A = __ldg(d.cov_atom + e);
                    const Four<T> g = load4(d.cov_gam + 4 * (int64_t)e);
                    const Four<T> c4 = load4(cproj + ((int64_t)A * nb + sg0 + s) * 4);
                    out += g.a * c4.a + g.b * c4.b + g.c * c4.c + g.d * c4.d;
                }
                hpsi[(int64_t)r * ldh + sg0 + s] = out;
            }

#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
#pragma unroll
                for (int k = 0; k < 8; ++k) q[dy][dx][k] = q[dy][dx][k + 1];
                q[dy][dx][8] = nq[dy][dx];
            }
        halo_rows(z + 3);
        slot = slot == 2 ? 0 : slot + 1;
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ------------------------------- FP32 kernel with per-chunk NL staging ---
// The same march as k_stencil for FP32 blocks of 32 states on 8 x 8 tiles, with
// everything irregular about a work item staged in shared memory once, at its
// start: interior and halo point rows, each output point's potential, and the
// nonlocal entries (projector values and atom) of all its output points (the
// host bounds the entries of a work item by V3_CAP).  In the march the only
// global traffic is psi (queue refill, halo copies), the projection
// coefficients (L1-resident) and the H psi stores.

constexpr int V3_CAP = 3584;   // nonlocal entries per work item
constexpr int V3_TX = 8, V3_TY = 8, V3_SG = 32;

struct V3Cfg {
    static constexpr int TX = V3_TX, TY = V3_TY, SG = V3_SG;
    static constexpr int W2 = TX + 8, W1 = TY + 8;
    static constexpr int PLANE = W1 * W2 * SG;
    static constexpr int NT = (TX / 2) * (TY / 2) * SG;   // 512
    static constexpr int RING = 3;
    static constexpr int CPR = 8;                          // 16-byte copies per 128-byte row
    static constexpr int NH = 8 * TY + 8 * TX;
    static constexpr int HPT = (NH * CPR + NT - 1) / NT;
    static constexpr int NI = TX * TY;
    static constexpr size_t OFF_ROWS = (size_t)RING * PLANE * 4;
    static constexpr size_t OFF_HROWS = OFF_ROWS + (size_t)(ZCHUNK + 9) * NI * 4;
    static constexpr size_t OFF_PV = OFF_HROWS + (size_t)ZCHUNK * NH * 4;
    static constexpr size_t OFF_PE = OFF_PV + (size_t)ZCHUNK * NI * 4;
    static constexpr size_t OFF_EG = OFF_PE + (size_t)ZCHUNK * NI * 4;
    static constexpr size_t OFF_EA = OFF_EG + (size_t)V3_CAP * 16;
    static constexpr size_t OFF_SCAN = OFF_EA + (size_t)V3_CAP * 4;
    static constexpr size_t SMEM = OFF_SCAN + 32 * 4;
};

__global__ void __launch_bounds__(V3Cfg::NT, 1)
    k_stencil_v3(HamDev<float> d, const float *__restrict__ psi, int64_t ldp, float *__restrict__ hpsi, int64_t ldh,
                 const float *__restrict__ cproj, int nb, const int4 *__restrict__ work) {
    using C = V3Cfg;
    constexpr int TX = C::TX, TY = C::TY, SG = C::SG;
    extern __shared__ __align__(16) unsigned char smraw[];
    float *sm = reinterpret_cast<float *>(smraw);
    int *rows = reinterpret_cast<int *>(smraw + C::OFF_ROWS);
    int *hrows = reinterpret_cast<int *>(smraw + C::OFF_HROWS);
    float *pv = reinterpret_cast<float *>(smraw + C::OFF_PV);
    int *pe = reinterpret_cast<int *>(smraw + C::OFF_PE);
    float4 *eg = reinterpret_cast<float4 *>(smraw + C::OFF_EG);
    int *ea = reinterpret_cast<int *>(smraw + C::OFF_EA);
    int *wsum = reinterpret_cast<int *>(smraw + C::OFF_SCAN);

    const int tid = threadIdx.x;
    const int s = tid % SG;
    const int patch = tid / SG;
    const int lx = 2 * (patch % (TX / 2));
    const int ly = 2 * (patch / (TX / 2));
    const int4 wk = work[blockIdx.x];
    const int b1 = wk.x * TY, b2 = wk.y * TX;
    const int za = wk.z, zb = wk.w;
    const int nz = zb - za;
    const int sg0 = blockIdx.y * SG;
    const float *psig = psi + sg0;

    auto map_at = [&](int a0, int a1, int a2) -> int {
        if ((unsigned)a0 >= (unsigned)d.d0 || (unsigned)a1 >= (unsigned)d.d1 || (unsigned)a2 >= (unsigned)d.d2)
            return -1;
        return __ldg(d.map + ((int64_t)a0 * d.d1 + a1) * d.d2 + a2);
    };
    auto halo_pos = [&](int hh, int &hy, int &hx) {
        if (hh < 8 * TY) {
            hy = hh >> 3;
            const int t = hh & 7;
            hx = t < 4 ? t - 4 : TX + t - 4;
        } else {
            const int h2 = hh - 8 * TY;
            hx = h2 % TX;
            const int t = h2 / TX;
            hy = t < 4 ? t - 4 : TY + t - 4;
        }
    };

    // ---- stage the work item's rows
    for (int e = tid; e < (nz + 9) * C::NI; e += C::NT) {
        const int pl = e / C::NI, pos = e % C::NI;
        rows[e] = map_at(za - 4 + pl, b1 + pos / TX, b2 + pos % TX);
    }
    for (int e = tid; e < nz * C::NH; e += C::NT) {
        int hy, hx;
        halo_pos(e % C::NH, hy, hx);
        hrows[e] = map_at(za + e / C::NH, b1 + hy, b2 + hx);
    }
    __syncthreads();
    // ---- potential and nonlocal entry counts of the output points; exclusive scan
    constexpr int PPT = ZCHUNK * C::NI / C::NT;   // output points per thread (4)
    int cnt[PPT], e0[PPT], tot = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int lp = tid * PPT + k;
        cnt[k] = 0;
        e0[k] = 0;
        float v = 0.f;
        if (lp < nz * C::NI) {
            const int r = rows[(lp / C::NI + 4) * C::NI + lp % C::NI];
            if (r >= 0) {
                const int4 inf = __ldg(d.pinfo + r);
                e0[k] = inf.x;
                cnt[k] = inf.y - inf.x;
                v = __int_as_float(inf.z);
            }
            pv[lp] = v;
        }
        tot += cnt[k];
    }
    // block-wide exclusive scan of tot
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((tid & 31) >= o) incl += y;
    }
    if ((tid & 31) == 31) wsum[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        int x = tid < C::NT / 32 ? wsum[tid] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (tid >= o) x += y;
        }
        wsum[tid] = x;  // inclusive per-warp totals
    }
    __syncthreads();
    int start = incl - tot + ((tid >> 5) ? wsum[(tid >> 5) - 1] : 0);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int lp = tid * PPT + k;
        if (lp < nz * C::NI) pe[lp] = (start << 4) | cnt[k];
        for (int j = 0; j < cnt[k]; ++j) {
            if (start + j < V3_CAP) {
                const float4 gv = __ldg(reinterpret_cast<const float4 *>(d.cov_gam) + e0[k] + j);
                eg[start + j] = gv;
                ea[start + j] = __ldg(d.cov_atom + e0[k] + j) * nb;
            }
        }
        start += cnt[k];
    }

    auto row_of = [&](int z, int iy, int ix) -> int { return rows[(z - za + 4) * C::NI + iy * TX + ix]; };
    auto load_val = [&](int r) -> float { return r >= 0 ? __ldg(psig + (int64_t)r * ldp + s) : 0.f; };
    auto issue_halo = [&](int z, int slot) {
        float *base = sm + slot * C::PLANE;
        const int *hr = hrows + (z - za) * C::NH;
#pragma unroll
        for (int j = 0; j < C::HPT; ++j) {
            const int i = tid + j * C::NT;
            if (i >= C::NH * C::CPR) continue;
            const int hh = i / C::CPR, c = i % C::CPR;
            int hy, hx;
            halo_pos(hh, hy, hx);
            const int r = hr[hh];
            const float *src = r >= 0 ? psig + (int64_t)r * ldp + c * 4 : psig;
            cp_async<16>(base + ((hy + 4) * C::W2 + (hx + 4)) * SG + c * 4, src, r >= 0);
        }
    };
    __syncthreads();

    float q[2][2][9];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) q[dy][dx][k] = load_val(row_of(za - 4 + k, ly + dy, lx + dx));
    issue_halo(za, 0);
    cp_async_commit();
    if (za + 1 < zb) issue_halo(za + 1, 1);
    cp_async_commit();

    const float w0 = d.w[0], w1 = d.w[1], w2 = d.w[2], w3 = d.w[3], w4 = d.w[4];
    const float *cpl = cproj + (int64_t)(sg0 + s) * 4;
    int slot = 0;
    for (int z = za; z < zb; ++z) {
        const int pslot = slot == 0 ? 2 : slot - 1;
        if (z + 2 < zb) issue_halo(z + 2, pslot);
        cp_async_commit();
        float nq[2][2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) nq[dy][dx] = load_val(row_of(z + 5, ly + dy, lx + dx));
        float *P = sm + slot * C::PLANE;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) P[((ly + dy + 4) * C::W2 + lx + dx + 4) * SG + s] = q[dy][dx][4];
        cp_async_wait<2>();
        __syncthreads();

        float acc[2][2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx)
                acc[dy][dx] = w0 * q[dy][dx][4] + w1 * (q[dy][dx][5] + q[dy][dx][3]) + w2 * (q[dy][dx][6] + q[dy][dx][2]) +
                              w3 * (q[dy][dx][7] + q[dy][dx][1]) + w4 * (q[dy][dx][8] + q[dy][dx][0]);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            float v[10];
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (k != 4 && k != 5) v[k] = P[((ly + dy + 4) * C::W2 + lx + k) * SG + s];
            v[4] = q[dy][0][4];
            v[5] = q[dy][1][4];
#pragma unroll
            for (int dx = 0; dx < 2; ++dx)
                acc[dy][dx] += w1 * (v[5 + dx] + v[3 + dx]) + w2 * (v[6 + dx] + v[2 + dx]) + w3 * (v[7 + dx] + v[1 + dx]) +
                               w4 * (v[8 + dx] + v[0 + dx]);
        }
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            float v[10];
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (k != 4 && k != 5) v[k] = P[((ly + k) * C::W2 + lx + dx + 4) * SG + s];
            v[4] = q[0][dx][4];
            v[5] = q[1][dx][4];
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
                acc[dy][dx] += w1 * (v[5 + dy] + v[3 + dy]) + w2 * (v[6 + dy] + v[2 + dy]) + w3 * (v[7 + dy] + v[1 + dy]) +
                               w4 * (v[8 + dy] + v[0 + dy]);
        }
        const int pbase = (z - za) * C::NI;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int pos = (ly + dy) * TX + lx + dx;
                const int r = rows[(z - za + 4) * C::NI + pos];
                if (r < 0) continue;
                const int code = pe[pbase + pos];
                float out = acc[dy][dx] + pv[pbase + pos] * q[dy][dx][4];
                const int e1 = min((code >> 4) + (code & 15), V3_CAP);
                for (int e = code >> 4; e < e1; ++e) {
                    const float4 gv = eg[e];
                    const float4 c4 = __ldg(reinterpret_cast<const float4 *>(cpl + (int64_t)ea[e] * 4) );
                    out += gv.x * c4.x + gv.y * c4.y + gv.z * c4.z + gv.w * c4.w;
                }
                hpsi[(int64_t)r * ldh + sg0 + s] = out;
            }
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
#pragma unroll
                for (int k = 0; k < 8; ++k) q[dy][dx][k] = q[dy][dx][k + 1];
                q[dy][dx][8] = nq[dy][dx];
            }
        slot = slot == 2 ? 0 : slot + 1;
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ------------------------- FP32 kernel v4: two states per lane, packed FMA ---
// Same work items and staging as k_stencil_v3, but every lane owns two
// adjacent states (a float2) so that the stencil runs on the packed FP32x2
// pipes (one FFMA2 / FADD2 per two outputs) and each shared-memory or global
// access moves 8 bytes; 16 lanes cover a point's 32 states and a warp two
// 2 x 2 patches.  The 9-deep plane queue is rotated by unrolling the march
// nine times instead of moving registers.

struct V4Cfg {
    static constexpr int TX = V3_TX, TY = V3_TY, SG = V3_SG;
    static constexpr int W2 = TX + 8, W1 = TY + 8;
    static constexpr int PLANE = W1 * W2 * SG;
    static constexpr int NT = (TX / 2) * (TY / 2) * (SG / 2);   // 256
    static constexpr int RING = 3;
    static constexpr int CPR = 8;
    static constexpr int NH = 8 * TY + 8 * TX;
    static constexpr int HPT = (NH * CPR + NT - 1) / NT;       // 4
    static constexpr int NI = TX * TY;
    static constexpr size_t OFF_ROWS = (size_t)RING * PLANE * 4;
    static constexpr size_t OFF_HROWS = OFF_ROWS + (size_t)(ZCHUNK + 9) * NI * 4;
    static constexpr size_t OFF_PV = OFF_HROWS + (size_t)ZCHUNK * NH * 4;
    static constexpr size_t OFF_PE = OFF_PV + (size_t)ZCHUNK * NI * 4;
    static constexpr size_t OFF_EG = OFF_PE + (size_t)ZCHUNK * NI * 4;
    static constexpr size_t OFF_EA = OFF_EG + (size_t)V3_CAP * 16;
    static constexpr size_t OFF_SCAN = OFF_EA + (size_t)V3_CAP * 4;
    static constexpr size_t SMEM = OFF_SCAN + 32 * 4;
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pair_sum(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int N> struct IC { static constexpr int value = N; };

__global__ void __launch_bounds__(V4Cfg::NT, 1)
    k_stencil_v4(HamDev<float> d, const float *__restrict__ psi, int64_t ldp, float *__restrict__ hpsi, int64_t ldh,
                 const float *__restrict__ cproj, int nb, const int4 *__restrict__ work) {
    using C = V4Cfg;
    constexpr int TX = C::TX, TY = C::TY, SG = C::SG;
    extern __shared__ __align__(16) unsigned char smraw[];
    float *sm = reinterpret_cast<float *>(smraw);
    int *rows = reinterpret_cast<int *>(smraw + C::OFF_ROWS);
    int *hrows = reinterpret_cast<int *>(smraw + C::OFF_HROWS);
    float *pv = reinterpret_cast<float *>(smraw + C::OFF_PV);
    int *pe = reinterpret_cast<int *>(smraw + C::OFF_PE);
    float4 *eg = reinterpret_cast<float4 *>(smraw + C::OFF_EG);
    int *ea = reinterpret_cast<int *>(smraw + C::OFF_EA);
    int *wsum = reinterpret_cast<int *>(smraw + C::OFF_SCAN);

    const int tid = threadIdx.x;
    const int s2 = tid % (SG / 2);          // state pair: states 2 s2, 2 s2 + 1 of the group
    const int patch = tid / (SG / 2);
    const int lx = 2 * (patch % (TX / 2));
    const int ly = 2 * (patch / (TX / 2));
    const int4 wk = work[blockIdx.x];
    const int b1 = wk.x * TY, b2 = wk.y * TX;
    const int za = wk.z, zb = wk.w;
    const int nz = zb - za;
    const int sg0 = blockIdx.y * SG;
    const float *psig = psi + sg0;

    auto map_at = [&](int a0, int a1, int a2) -> int {
        if ((unsigned)a0 >= (unsigned)d.d0 || (unsigned)a1 >= (unsigned)d.d1 || (unsigned)a2 >= (unsigned)d.d2)
            return -1;
        return __ldg(d.map + ((int64_t)a0 * d.d1 + a1) * d.d2 + a2);
    };
    auto halo_pos = [&](int hh, int &hy, int &hx) {
        if (hh < 8 * TY) {
            hy = hh >> 3;
            const int t = hh & 7;
            hx = t < 4 ? t - 4 : TX + t - 4;
        } else {
            const int h2 = hh - 8 * TY;
            hx = h2 % TX;
            const int t = h2 / TX;
            hy = t < 4 ? t - 4 : TY + t - 4;
        }
    };

    // ---- stage the work item (as in k_stencil_v3)
    for (int e = tid; e < (nz + 9) * C::NI; e += C::NT) {
        const int pl = e / C::NI, pos = e % C::NI;
        rows[e] = map_at(za - 4 + pl, b1 + pos / TX, b2 + pos % TX);
    }
    for (int e = tid; e < nz * C::NH; e += C::NT) {
        int hy, hx;
        halo_pos(e % C::NH, hy, hx);
        hrows[e] = map_at(za + e / C::NH, b1 + hy, b2 + hx);
    }
    __syncthreads();
    constexpr int PPT = ZCHUNK * C::NI / C::NT;   // 8
    int cnt[PPT], e0[PPT], tot = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int lp = tid * PPT + k;
        cnt[k] = 0;
        e0[k] = 0;
        float v = 0.f;
        if (lp < nz * C::NI) {
            const int r = rows[(lp / C::NI + 4) * C::NI + lp % C::NI];
            if (r >= 0) {
                const int4 inf = __ldg(d.pinfo + r);
                e0[k] = inf.x;
                cnt[k] = inf.y - inf.x;
                v = __int_as_float(inf.z);
            }
            pv[lp] = v;
        }
        tot += cnt[k];
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((tid & 31) >= o) incl += y;
    }
    if ((tid & 31) == 31) wsum[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        int x = tid < C::NT / 32 ? wsum[tid] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (tid >= o) x += y;
        }
        wsum[tid] = x;
    }
    __syncthreads();
    int start = incl - tot + ((tid >> 5) ? wsum[(tid >> 5) - 1] : 0);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int lp = tid * PPT + k;
        if (lp < nz * C::NI) pe[lp] = (start << 4) | cnt[k];
        for (int j = 0; j < cnt[k]; ++j) {
            if (start + j < V3_CAP) {
                eg[start + j] = __ldg(reinterpret_cast<const float4 *>(d.cov_gam) + e0[k] + j);
                ea[start + j] = __ldg(d.cov_atom + e0[k] + j) * nb;
            }
        }
        start += cnt[k];
    }
    __syncthreads();

    auto row_of = [&](int z, int iy, int ix) -> int { return rows[(z - za + 4) * C::NI + iy * TX + ix]; };
    auto load2 = [&](int r) -> float2 {
        return r >= 0 ? __ldg(reinterpret_cast<const float2 *>(psig + (int64_t)r * ldp) + s2) : make_float2(0.f, 0.f);
    };
    auto issue_halo = [&](int z, int slot) {
        float *base = sm + slot * C::PLANE;
        const int *hr = hrows + (z - za) * C::NH;
#pragma unroll
        for (int j = 0; j < C::HPT; ++j) {
            const int i = tid + j * C::NT;
            if (i >= C::NH * C::CPR) continue;
            const int hh = i / C::CPR, c = i % C::CPR;
            int hy, hx;
            halo_pos(hh, hy, hx);
            const int r = hr[hh];
            const float *src = r >= 0 ? psig + (int64_t)r * ldp + c * 4 : psig;
            cp_async<16>(base + ((hy + 4) * C::W2 + (hx + 4)) * SG + c * 4, src, r >= 0);
        }
    };

    float2 q[2][2][9];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) q[dy][dx][k] = load2(row_of(za - 4 + k, ly + dy, lx + dx));
    issue_halo(za, 0);
    cp_async_commit();
    if (za + 1 < zb) issue_halo(za + 1, 1);
    cp_async_commit();

    const float2 W0 = f2(d.w[0]), W1 = f2(d.w[1]), W2 = f2(d.w[2]), W3 = f2(d.w[3]), W4 = f2(d.w[4]);
    const float *cpl = cproj + (int64_t)(sg0 + 2 * s2) * 4;
    int slot = 0;
    // one plane of the march; queue slot of plane z + j is (j + 4 + R) % 9
    auto step = [&](int z, auto Rc) {
        constexpr int R = decltype(Rc)::value;
#define QS(dy, dx, j) q[dy][dx][((j) + 4 + R) % 9]
        const int pslot = slot == 0 ? 2 : slot - 1;
        if (z + 2 < zb) issue_halo(z + 2, pslot);
        cp_async_commit();
        float2 nq[2][2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) nq[dy][dx] = load2(row_of(z + 5, ly + dy, lx + dx));
        float *P = sm + slot * C::PLANE;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx)
                reinterpret_cast<float2 *>(P + ((ly + dy + 4) * C::W2 + lx + dx + 4) * SG)[s2] = QS(dy, dx, 0);
        cp_async_wait<2>();
        __syncthreads();

        float2 acc[2][2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                float2 a = __fmul2_rn(W0, QS(dy, dx, 0));
                a = fma2(W1, pair_sum(QS(dy, dx, 1), QS(dy, dx, -1)), a);
                a = fma2(W2, pair_sum(QS(dy, dx, 2), QS(dy, dx, -2)), a);
                a = fma2(W3, pair_sum(QS(dy, dx, 3), QS(dy, dx, -3)), a);
                a = fma2(W4, pair_sum(QS(dy, dx, 4), QS(dy, dx, -4)), a);
                acc[dy][dx] = a;
            }
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            float2 v[10];
            const float2 *row = reinterpret_cast<const float2 *>(P + ((ly + dy + 4) * C::W2 + lx) * SG) + s2;
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (k != 4 && k != 5) v[k] = row[k * (SG / 2)];
            v[4] = QS(dy, 0, 0);
            v[5] = QS(dy, 1, 0);
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                float2 a = acc[dy][dx];
                a = fma2(W1, pair_sum(v[5 + dx], v[3 + dx]), a);
                a = fma2(W2, pair_sum(v[6 + dx], v[2 + dx]), a);
                a = fma2(W3, pair_sum(v[7 + dx], v[1 + dx]), a);
                a = fma2(W4, pair_sum(v[8 + dx], v[0 + dx]), a);
                acc[dy][dx] = a;
            }
        }
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            float2 v[10];
            const float2 *col = reinterpret_cast<const float2 *>(P + (ly * C::W2 + lx + dx + 4) * SG) + s2;
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (k != 4 && k != 5) v[k] = col[k * C::W2 * (SG / 2)];
            v[4] = QS(0, dx, 0);
            v[5] = QS(1, dx, 0);
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                float2 a = acc[dy][dx];
                a = fma2(W1, pair_sum(v[5 + dy], v[3 + dy]), a);
                a = fma2(W2, pair_sum(v[6 + dy], v[2 + dy]), a);
                a = fma2(W3, pair_sum(v[7 + dy], v[1 + dy]), a);
                a = fma2(W4, pair_sum(v[8 + dy], v[0 + dy]), a);
                acc[dy][dx] = a;
            }
        }
        const int pbase = (z - za) * C::NI;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int pos = (ly + dy) * TX + lx + dx;
                const int r = rows[(z - za + 4) * C::NI + pos];
                if (r < 0) continue;
                const int code = pe[pbase + pos];
                float2 out = fma2(f2(pv[pbase + pos]), QS(dy, dx, 0), acc[dy][dx]);
                const int e1 = min((code >> 4) + (code & 15), V3_CAP);
                for (int e = code >> 4; e < e1; ++e) {
                    const float4 gv = eg[e];
                    const float4 *cp = reinterpret_cast<const float4 *>(cpl + (int64_t)ea[e] * 4);
                    const float4 ca = __ldg(cp), cb = __ldg(cp + 1);
                    out.x += gv.x * ca.x + gv.y * ca.y + gv.z * ca.z + gv.w * ca.w;
                    out.y += gv.x * cb.x + gv.y * cb.y + gv.z * cb.z + gv.w * cb.w;
                }
                reinterpret_cast<float2 *>(hpsi + (int64_t)r * ldh + sg0)[s2] = out;
            }
        // the oldest plane's slot receives plane z + 5 (it is plane z + 4 of the next step)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) QS(dy, dx, -4) = nq[dy][dx];
#undef QS
        slot = slot == 2 ? 0 : slot + 1;
        __syncthreads();
    };
    for (int z = za; z < zb; z += 9) {
        step(z, IC<0>{});
        if (z + 1 < zb) step(z + 1, IC<1>{}); else break;
        if (z + 2 < zb) step(z + 2, IC<2>{}); else break;
        if (z + 3 < zb) step(z + 3, IC<3>{}); else break;
        if (z + 4 < zb) step(z + 4, IC<4>{}); else break;
        if (z + 5 < zb) step(z + 5, IC<5>{}); else break;
        if (z + 6 < zb) step(z + 6, IC<6>{}); else break;
        if (z + 7 < zb) step(z + 7, IC<7>{}); else break;
        if (z + 8 < zb) step(z + 8, IC<8>{}); else break;
    }
    cp_async_wait<0>();
}

// ----------------------------------------------- face-neighbour filter ---
// W = alpha R + beta sum_{6 face neighbours} R (zero off the grid); one thread
// per (point, state), state fastest.
template <typename T>
__global__ void k_filter(const int32_t *__restrict__ map, const int32_t *__restrict__ loc, int64_t npts, int d1, int d2,
                         const T *__restrict__ R, int64_t ldr, T *__restrict__ W, int64_t ldw, int nb, T alpha,
                         T beta) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = t / nb;
    const int s = (int)(t % nb);
    if (p >= npts) return;
    const int64_t L = __ldg(loc + p);
    const int64_t plane = (int64_t)d1 * d2;
    const int64_t offs[6] = {1, -1, d2, -(int64_t)d2, plane, -plane};
    T acc = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int q = __ldg(map + L + offs[k]);
        if (q >= 0) acc += __ldg(R + (int64_t)q * ldr + s);
    }
    W[p * ldw + s] = alpha * __ldg(R + p * ldr + s) + beta * acc;
}

}  // namespace rs

using namespace rs;

// ------------------------------------------------------------ host side ---

namespace {

struct WorkList {
    DevBuf buf;
    int count = 0;
};

// Tile shapes (TX along map axis 2, TY along map axis 1) per state-group size.
struct Shape {
    int sg, tx, ty;
};
const Shape kShapes[] = {{32, 8, 8}, {16, 16, 8}, {8, 16, 16}, {4, 32, 16}, {2, 32, 32}, {1, 64, 32}};
const int kZChunk = ZCHUNK;

}  // namespace

struct rs_ham {
    int64_t npts = 0;
    int32_t d[3] = {0, 0, 0};
    double h = 0, dV = 0;
    int order = 4;
    int n_atoms = 0;
    int64_t n_entries = 0;
    int device = 0;
    double w[5] = {0, 0, 0, 0, 0};
    DevBuf pinfo64, pinfo32, map, loc, V64, V32, cov_off, cov_atom, cov_gam64, cov_gam32, sph_off, sph_idx, sph_gam64, sph_gam32, E64, E32,
        cproj, dummy, scratch;
    std::map<std::pair<int, int>, WorkList *> work;
    WorkList *work_v3 = nullptr;   // FP32 32-state kernel with bounded nonlocal entries per item
    RingPlan *ring = nullptr;      // tables of the ring-buffer FP32 kernel (nullptr: not usable)
    // optional per-launch timing (rs_ham_timing)
    bool timing = false;
    std::vector<cudaEvent_t> events;   // 3 per recorded call
    size_t n_recorded = 0;
    ~rs_ham() {
        ring_plan_destroy(ring);
        delete work_v3;
        for (auto &kv : work) delete kv.second;
        for (cudaEvent_t e : events) cudaEventDestroy(e);
    }
    // events for the next recorded call (nullptr when timing is off)
    cudaEvent_t *next_events() {
        if (!timing) return nullptr;
        if (events.size() < 3 * (n_recorded + 1)) {
            for (int i = 0; i < 3; ++i) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
                events.push_back(e);
            }
        }
        return &events[3 * n_recorded++];
    }
    template <typename T> HamDev<T> view() const;
};

template <> HamDev<double> rs_ham::view<double>() const {
    HamDev<double> v;
    v.pinfo = pinfo64.as<int4>();
    v.map = map.as<int32_t>();
    v.d0 = d[0], v.d1 = d[1], v.d2 = d[2];
    v.V = V64.as<double>();
    v.cov_off = cov_off.as<int32_t>();
    v.cov_atom = cov_atom.as<int32_t>();
    v.cov_gam = cov_gam64.as<double>();
    v.sph_off = sph_off.as<int32_t>();
    v.sph_idx = sph_idx.as<int32_t>();
    v.sph_gam = sph_gam64.as<double>();
    v.E = E64.as<double>();
    v.dV = dV;
    for (int j = 0; j < 5; ++j) v.w[j] = w[j];
    return v;
}
template <> HamDev<float> rs_ham::view<float>() const {
    HamDev<float> v;
    v.pinfo = pinfo32.as<int4>();
    v.map = map.as<int32_t>();
    v.d0 = d[0], v.d1 = d[1], v.d2 = d[2];
    v.V = V32.as<float>();
    v.cov_off = cov_off.as<int32_t>();
    v.cov_atom = cov_atom.as<int32_t>();
    v.cov_gam = cov_gam32.as<float>();
    v.sph_off = sph_off.as<int32_t>();
    v.sph_idx = sph_idx.as<int32_t>();
    v.sph_gam = sph_gam32.as<float>();
    v.E = E32.as<float>();
    v.dV = (float)dV;
    for (int j = 0; j < 5; ++j) v.w[j] = (float)w[j];
    return v;
}

// Central second-derivative weights of half-width m (closed form):
// c_j = 2 (-1)^(j+1) (m!)^2 / (j^2 (m-j)! (m+j)!), c_0 = -2 sum_{j>=1} c_j.
static void fd_weights(int m, double c[5]) {
    auto fact = [](int n) {
        double f = 1;
        for (int i = 2; i <= n; ++i) f *= i;
        return f;
    };
    for (int j = 0; j < 5; ++j) c[j] = 0;
    double sum = 0;
    for (int j = 1; j <= m; ++j) {
        c[j] = 2.0 * ((j & 1) ? 1.0 : -1.0) * fact(m) * fact(m) / ((double)j * j * fact(m - j) * fact(m + j));
        sum += c[j];
    }
    c[0] = -2.0 * sum;
}

static int build_work(rs_ham *H, const rs_grid *g, int tx, int ty) {
    const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
    const int n1 = (d1 + ty - 1) / ty, n2 = (d2 + tx - 1) / tx;
    std::vector<int> zmin((size_t)n1 * n2, d0), zmax((size_t)n1 * n2, -1);
    for (int a = 0; a < d0; ++a)
        for (int b = 0; b < d1; ++b)
            for (int c = 0; c < d2; ++c)
                if (g->map[((size_t)a * d1 + b) * d2 + c] >= 0) {
                    const size_t t = (size_t)(b / ty) * n2 + (c / tx);
                    zmin[t] = std::min(zmin[t], a);
                    zmax[t] = std::max(zmax[t], a);
                }
    std::vector<int4> items;
    for (int t1 = 0; t1 < n1; ++t1)
        for (int t2 = 0; t2 < n2; ++t2) {
            const size_t t = (size_t)t1 * n2 + t2;
            if (zmax[t] < 0) continue;
            for (int z = zmin[t]; z <= zmax[t]; z += kZChunk) items.push_back(make_int4(t1, t2, z, std::min(z + kZChunk, zmax[t] + 1)));
        }
    // raster order over (tile row, tile column, z chunk): CTAs resident at the
    // same time are spatial neighbours, so halo rows are re-read from L2
    WorkList *wl = new (std::nothrow) WorkList;
    if (!wl) return fail(RS_ENOMEM, "host allocation failed");
    H->work[{tx, ty}] = wl;
    wl->count = (int)items.size();
    return wl->buf.upload(items.data(), items.size() * sizeof(int4));
}

// Work items of k_stencil_v3: 8 x 8 tile columns cut into chunks of at most
// ZCHUNK planes and at most V3_CAP nonlocal entries.  Returns false (no list)
// when some point is covered by more than 15 projector spheres.
static int build_work_v3(rs_ham *H, const rs_grid *g, const std::vector<int32_t> &coff, bool *ok) {
    const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
    const int tx = V3_TX, ty = V3_TY;
    *ok = false;
    for (int64_t p = 0; p < g->npts; ++p)
        if (coff[p + 1] - coff[p] > 15) return RS_OK;
    const int n1 = (d1 + ty - 1) / ty, n2 = (d2 + tx - 1) / tx;
    std::vector<int4> items;
    for (int t1 = 0; t1 < n1; ++t1)
        for (int t2 = 0; t2 < n2; ++t2) {
            int za = -1, entries = 0;
            for (int a = 0; a < d0; ++a) {
                int e = 0, any = 0;
                for (int b = t1 * ty; b < std::min(d1, (t1 + 1) * ty); ++b)
                    for (int c = t2 * tx; c < std::min(d2, (t2 + 1) * tx); ++c) {
                        const int32_t p = g->map[((size_t)a * d1 + b) * d2 + c];
                        if (p >= 0) {
                            any = 1;
                            e += coff[p + 1] - coff[p];
                        }
                    }
                if (za >= 0 && (a - za == ZCHUNK || entries + e > V3_CAP)) {
                    items.push_back(make_int4(t1, t2, za, a));
                    za = -1;
                    entries = 0;
                }
                if (any && za < 0) za = a;
                if (za >= 0) entries += e;
            }
            if (za >= 0) {
                // trim trailing empty planes
                int zb = d0;
                while (zb > za) {
                    bool any = false;
                    for (int b = t1 * ty; b < std::min(d1, (t1 + 1) * ty) && !any; ++b)
                        for (int c = t2 * tx; c < std::min(d2, (t2 + 1) * tx) && !any; ++c)
                            any = g->map[((size_t)(zb - 1) * d1 + b) * d2 + c] >= 0;
                    if (any) break;
                    --zb;
                }
                items.push_back(make_int4(t1, t2, za, zb));
            }
        }
    WorkList *wl = new (std::nothrow) WorkList;
    if (!wl) return fail(RS_ENOMEM, "host allocation failed");
    H->work_v3 = wl;
    wl->count = (int)items.size();
    *ok = true;
    return wl->buf.upload(items.data(), items.size() * sizeof(int4));
}

extern "C" int rs_ham_create(const rs_grid *g, const double *V_host, const rs_proj *pr, int order, rs_ham **out) {
    if (!g || !V_host || !out) return fail(RS_EINVAL, "rs_ham_create: null argument");
    if (order < 1 || order > 4) return fail(RS_EINVAL, "rs_ham_create: order must be in 1..4");
    *out = nullptr;
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    rs_ham *H = new (std::nothrow) rs_ham;
    if (!H) return fail(RS_ENOMEM, "host allocation failed");
    auto bail = [&](int rc) {
        delete H;
        return rc;
    };
    H->device = dev;
    H->npts = g->npts;
    for (int i = 0; i < 3; ++i) H->d[i] = g->dims[i];
    H->h = g->h;
    H->dV = g->h * g->h * g->h;
    H->order = order;
    double c[5];
    fd_weights(order, c);
    const double kin = -0.5 / (g->h * g->h);
    H->w[0] = 3.0 * kin * c[0];
    for (int j = 1; j < 5; ++j) H->w[j] = kin * c[j];

    int rc;
    const int64_t np = g->npts;
    if ((rc = H->map.upload(g->map.data(), g->map.size() * sizeof(int32_t)))) return bail(rc);
    {
        std::vector<int32_t> loc((size_t)g->npts);
        for (int64_t p = 0; p < g->npts; ++p)
            loc[p] = (int32_t)(((int64_t)(g->ijk[3 * p] - g->origin[0]) * g->dims[1] + (g->ijk[3 * p + 1] - g->origin[1])) *
                                   g->dims[2] + (g->ijk[3 * p + 2] - g->origin[2]));
        if ((rc = H->loc.upload(loc.data(), loc.size() * sizeof(int32_t)))) return bail(rc);
    }
    std::vector<float> v32((size_t)np);
    for (int64_t p = 0; p < np; ++p) v32[p] = (float)V_host[p];
    if ((rc = H->V64.upload(V_host, (size_t)np * sizeof(double)))) return bail(rc);
    if ((rc = H->V32.upload(v32.data(), (size_t)np * sizeof(float)))) return bail(rc);

    // projector tables: atom-major (projection) and point-major (gather)
    const int na = pr ? pr->n_atoms : 0;
    const int64_t ne = pr ? (int64_t)pr->idx.size() : 0;
    if (ne > (int64_t)INT32_MAX) return bail(fail(RS_EINVAL, "too many projector entries"));
    H->n_atoms = na;
    H->n_entries = ne;
    std::vector<int32_t> soff((size_t)na + 1, 0), coff((size_t)np + 1, 0), catom((size_t)std::max<int64_t>(ne, 1));
    std::vector<double> cg64((size_t)std::max<int64_t>(ne, 1) * 4), sg64((size_t)std::max<int64_t>(ne, 1) * 4),
        E64((size_t)std::max(na, 1) * 4);
    for (int A = 0; A < na; ++A) soff[A + 1] = (int32_t)pr->off[A + 1];
    for (int64_t e = 0; e < ne; ++e) coff[(size_t)pr->idx[e] + 1]++;
    for (int64_t p = 0; p < np; ++p) coff[p + 1] += coff[p];
    {
        std::vector<int32_t> fill(coff.begin(), coff.end() - 1);
        for (int A = 0; A < na; ++A)
            for (int64_t e = pr->off[A]; e < pr->off[A + 1]; ++e) {
                const int32_t slot = fill[pr->idx[e]]++;
                catom[slot] = A;
                for (int q = 0; q < 4; ++q) cg64[(size_t)slot * 4 + q] = pr->gam[e * 4 + q];
            }
    }
    for (int64_t e = 0; e < ne * 4; ++e) sg64[e] = pr->gam[e];
    for (int A = 0; A < na * 4; ++A) E64[A] = pr->E[A];
    std::vector<float> cg32(cg64.begin(), cg64.end()), sg32(sg64.begin(), sg64.end()), E32(E64.begin(), E64.end());
    std::vector<int32_t> sidx(pr && ne ? pr->idx : std::vector<int32_t>(1, 0));
    if ((rc = H->sph_off.upload(soff.data(), soff.size() * 4)) || (rc = H->sph_idx.upload(sidx.data(), sidx.size() * 4)) ||
        (rc = H->sph_gam64.upload(sg64.data(), sg64.size() * 8)) ||
        (rc = H->sph_gam32.upload(sg32.data(), sg32.size() * 4)) || (rc = H->E64.upload(E64.data(), E64.size() * 8)) ||
        (rc = H->E32.upload(E32.data(), E32.size() * 4)) || (rc = H->cov_off.upload(coff.data(), coff.size() * 4)) ||
        (rc = H->cov_atom.upload(catom.data(), catom.size() * 4)) ||
        (rc = H->cov_gam64.upload(cg64.data(), cg64.size() * 8)) ||
        (rc = H->cov_gam32.upload(cg32.data(), cg32.size() * 4)))
        return bail(rc);
    if ((rc = H->cproj.alloc((size_t)std::max(na, 1) * 4 * 64 * sizeof(double)))) return bail(rc);
    {
        std::vector<int4> p64((size_t)np), p32((size_t)np);
        for (int64_t p = 0; p < np; ++p) {
            int64_t bits;
            memcpy(&bits, &V_host[p], 8);
            int32_t fbits;
            memcpy(&fbits, &v32[p], 4);
            p64[p] = make_int4(coff[p], coff[p + 1], (int32_t)(bits & 0xffffffffll), (int32_t)(bits >> 32));
            p32[p] = make_int4(coff[p], coff[p + 1], fbits, 0);
        }
        if ((rc = H->pinfo64.upload(p64.data(), p64.size() * sizeof(int4))) ||
            (rc = H->pinfo32.upload(p32.data(), p32.size() * sizeof(int4))))
            return bail(rc);
    }
    for (const Shape &s : kShapes)
        if ((rc = build_work(H, g, s.tx, s.ty))) return bail(rc);
    bool v3ok = false;
    if ((rc = build_work_v3(H, g, coff, &v3ok))) return bail(rc);
#if RS_STENCIL_RING
    if ((rc = ring_plan_build(&H->ring, g, coff, catom, cg32, v32, na, RS_RING_SLAB))) return bail(rc);
#endif
    *out = H;
    return RS_OK;
}

extern "C" int rs_ham_destroy(rs_ham *h) {
    delete h;
    return RS_OK;
}

template <typename T, int SG, int TX, int TY>
static int launch_stencil(rs_ham *H, const HamDev<T> &d, const T *psi, int64_t ldp, T *hpsi, int64_t ldh, int nb,
                          cudaStream_t st) {
    using C = StencilCfg<T, SG, TX, TY>;
    static bool attr_done = false;  // per instantiation; set once per process
    if (!attr_done) {
        RS_CUDA(cudaFuncSetAttribute(k_stencil<T, SG, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        attr_done = true;
    }
    const WorkList *wl = H->work.at({TX, TY});
    if (wl->count == 0) return RS_OK;
    dim3 grid((unsigned)wl->count, (unsigned)(nb / SG));
    k_stencil<T, SG, TX, TY><<<grid, C::NT, C::SMEM, st>>>(d, psi, ldp, hpsi, ldh, H->cproj.as<T>(), nb,
                                                            wl->buf.as<int4>());
    RS_LAUNCH_CHECK();
    return RS_OK;
}

template <typename T>
static int launch_v3(rs_ham *H, const HamDev<T> &d, const T *psi, int64_t ldp, T *hpsi, int64_t ldh, int nb,
                     cudaStream_t st) {
    if constexpr (sizeof(T) != 4) {
        return fail(RS_EINVAL, "launch_v3: FP32 only");
    } else {
        const WorkList *wl = H->work_v3;
        if (wl->count == 0) return RS_OK;
        dim3 grid((unsigned)wl->count, (unsigned)(nb / V3_SG));
#if RS_STENCIL_V3
        static bool attr_done = false;
        if (!attr_done) {
            RS_CUDA(cudaFuncSetAttribute(k_stencil_v3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V3Cfg::SMEM));
            attr_done = true;
        }
        k_stencil_v3<<<grid, V3Cfg::NT, V3Cfg::SMEM, st>>>(d, psi, ldp, hpsi, ldh, H->cproj.as<T>(), nb, wl->buf.as<int4>());
#else
        static bool attr_done = false;
        if (!attr_done) {
            RS_CUDA(cudaFuncSetAttribute(k_stencil_v4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V4Cfg::SMEM));
            attr_done = true;
        }
        k_stencil_v4<<<grid, V4Cfg::NT, V4Cfg::SMEM, st>>>(d, psi, ldp, hpsi, ldh, H->cproj.as<T>(), nb, wl->buf.as<int4>());
#endif
        RS_LAUNCH_CHECK();
        return RS_OK;
    }
}

template <typename T>
static int apply_t(rs_ham *H, const T *psi, int64_t ldp, T *hpsi, int64_t ldh, int nb, cudaStream_t st) {
    const HamDev<T> d = H->view<T>();
    cudaEvent_t *ev = H->next_events();
    if (ev) RS_CUDA(cudaEventRecord(ev[0], st));
    if (H->n_atoms > 0) {
        const int sgp = std::min(nb, 32);
        dim3 grid((unsigned)(H->n_atoms * PSPLIT), (unsigned)(nb / sgp));
        T *cp = H->cproj.as<T>();
        RS_CUDA(cudaMemsetAsync(cp, 0, sizeof(T) * (size_t)H->n_atoms * 4 * nb, st));
        switch (sgp) {
            case 1: k_project<T, 1, 512><<<grid, 512, 0, st>>>(d, psi, ldp, nb, cp); break;
            case 2: k_project<T, 2, 512><<<grid, 512, 0, st>>>(d, psi, ldp, nb, cp); break;
            case 4: k_project<T, 4, 512><<<grid, 512, 0, st>>>(d, psi, ldp, nb, cp); break;
            case 8: k_project<T, 8, 512><<<grid, 512, 0, st>>>(d, psi, ldp, nb, cp); break;
            case 16: k_project<T, 16, 512><<<grid, 512, 0, st>>>(d, psi, ldp, nb, cp); break;
            default: k_project<T, 32, 512><<<grid, 512, 0, st>>>(d, psi, ldp, nb, cp); break;
        }
        RS_LAUNCH_CHECK();
    }
    if (ev) RS_CUDA(cudaEventRecord(ev[1], st));
    constexpr int SGMAX = 128 / (int)sizeof(T);
    const int sg = std::min(nb, SGMAX);
    int rc;
    switch (sg) {
        case 1: rc = launch_stencil<T, 1, 64, 32>(H, d, psi, ldp, hpsi, ldh, nb, st); break;
        case 2: rc = launch_stencil<T, 2, 32, 32>(H, d, psi, ldp, hpsi, ldh, nb, st); break;
        case 4: rc = launch_stencil<T, 4, 32, 16>(H, d, psi, ldp, hpsi, ldh, nb, st); break;
        case 8: rc = launch_stencil<T, 8, 16, 16>(H, d, psi, ldp, hpsi, ldh, nb, st); break;
        case 16: rc = launch_stencil<T, 16, 16, 8>(H, d, psi, ldp, hpsi, ldh, nb, st); break;
        default:
            if constexpr (SGMAX >= 32) {
                if constexpr (sizeof(T) == 4) {
                    if (ring_usable(H->ring, psi, ldp, nb)) {
                        float w[5];
                        for (int j = 0; j < 5; ++j) w[j] = (float)H->w[j];
                        rc = ring_launch(H->ring, psi, ldp, hpsi, ldh, H->cproj.as<float>(), nb, w, st);
                        break;
                    }
                }
                if (H->work_v3) {
                    rc = launch_v3(H, d, psi, ldp, hpsi, ldh, nb, st);
                    break;
                }
                rc = launch_stencil<T, 32, 8, 8>(H, d, psi, ldp, hpsi, ldh, nb, st);
                break;
            }
            return fail(RS_EINVAL, "unsupported state group");
    }
    if (rc == RS_OK && ev) RS_CUDA(cudaEventRecord(ev[2], st));
    return rc;
}

extern "C" int rs_ham_apply_block(rs_ham *h, const void *psi_dev, int64_t ld_psi, void *hpsi_dev, int64_t ld_hpsi,
                                  int nb, int dtype, void *stream) {
    if (!h || !psi_dev || !hpsi_dev) return fail(RS_EINVAL, "rs_ham_apply_block: null argument");
    if (nb < 1 || nb > 64 || (nb & (nb - 1))) return fail(RS_EINVAL, "rs_ham_apply_block: nb must be a power of two <= 64");
    if (ld_psi < nb || ld_hpsi < nb) return fail(RS_EINVAL, "rs_ham_apply_block: ld < nb");
    if (dtype != RS_F64 && dtype != RS_F32) return fail(RS_EINVAL, "rs_ham_apply_block: bad dtype");
    const int es = dtype == RS_F64 ? 8 : 4;
    const int sgbytes = std::min(nb, 128 / es) * es;
    const int need = std::min(sgbytes, 16);
    if (((uintptr_t)psi_dev % need) || ((uintptr_t)hpsi_dev % need) || ((ld_psi * es) % need) || ((ld_hpsi * es) % need))
        return fail(RS_EINVAL, "rs_ham_apply_block: misaligned pointer or leading dimension");
    const char *a = (const char *)psi_dev, *b = (const char *)hpsi_dev;
    const int64_t span_a = ((h->npts - 1) * ld_psi + nb) * es, span_b = ((h->npts - 1) * ld_hpsi + nb) * es;
    if (a < b + span_b && b < a + span_a) return fail(RS_EINVAL, "rs_ham_apply_block: psi and hpsi overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == RS_F64)
        return apply_t<double>(h, (const double *)psi_dev, ld_psi, (double *)hpsi_dev, ld_hpsi, nb, st);
    return apply_t<float>(h, (const float *)psi_dev, ld_psi, (float *)hpsi_dev, ld_hpsi, nb, st);
}

extern "C" int64_t rs_ham_apply_bytes(const rs_ham *h, int nb, int dtype) {
    int64_t a = 0, b = 0;
    if (rs_ham_launch_bytes(h, nb, dtype, &a, &b) != RS_OK) return -1;
    return a + b;
}

extern "C" int rs_ham_launch_bytes(const rs_ham *h, int nb, int dtype, int64_t *project_bytes, int64_t *stencil_bytes) {
    if (!h) return fail(RS_EINVAL, "rs_ham_launch_bytes: null handle");
    const int64_t s = dtype == RS_F64 ? 8 : 4;
    const int64_t np = h->npts, ne = h->n_entries, nc = (int64_t)h->n_atoms * 4 * nb * s;
    if (project_bytes) *project_bytes = ne * (4 + 4 * s) + (h->n_atoms + 1) * 4 + nc;
    if (stencil_bytes) *stencil_bytes = np * nb * 2 * s + np * s + np * 4 + ne * (4 + 4 * s) + (np + 1) * 4 + nc;
    return RS_OK;
}

extern "C" int rs_ham_status(rs_ham *h, int *flags) {
    if (!h || !flags) return fail(RS_EINVAL, "rs_ham_status: null argument");
    int f = 0;
    RS_TRY(ring_status(h->ring, &f));
    *flags = f;
    return RS_OK;
}

extern "C" int rs_ham_timing(rs_ham *h, int enable) {
    if (!h) return fail(RS_EINVAL, "rs_ham_timing: null handle");
    if (enable) h->n_recorded = 0;
    h->timing = enable != 0;
    return RS_OK;
}

extern "C" int rs_ham_timing_read(rs_ham *h, double *project_ms, double *stencil_ms, int64_t *calls) {
    if (!h) return fail(RS_EINVAL, "rs_ham_timing_read: null handle");
    double pm = 0, sm = 0;
    for (size_t i = 0; i < h->n_recorded; ++i) {
        cudaEvent_t *e = &h->events[3 * i];
        RS_CUDA(cudaEventSynchronize(e[2]));
        float a = 0, b = 0;
        RS_CUDA(cudaEventElapsedTime(&a, e[0], e[1]));
        RS_CUDA(cudaEventElapsedTime(&b, e[1], e[2]));
        pm += a;
        sm += b;
    }
    if (project_ms) *project_ms = pm;
    if (stencil_ms) *stencil_ms = sm;
    if (calls) *calls = (int64_t)h->n_recorded;
    return RS_OK;
}

namespace rs {

int64_t ham_npts(const rs_ham *h) { return h->npts; }
const int32_t *ham_map(const rs_ham *h) { return h->map.as<int32_t>(); }
const int32_t *ham_loc(const rs_ham *h) { return h->loc.as<int32_t>(); }
int ham_dim(const rs_ham *h, int axis) { return h->d[axis]; }
DevBuf *ham_scratch(rs_ham *h, size_t bytes) {
    if (h->scratch.bytes >= bytes) return &h->scratch;
    if (h->scratch.alloc(bytes) != RS_OK) return nullptr;
    return &h->scratch;
}
double ham_dV(const rs_ham *h) { return h->dV; }

int ham_filter(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype, double alpha,
               cudaStream_t st) {
    const int64_t n = h->npts * nb;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const double beta = (1.0 - alpha) / 6.0;
    if (dtype == RS_F64)
        k_filter<double><<<blocks, 256, 0, st>>>(h->map.as<int32_t>(), h->loc.as<int32_t>(), h->npts, h->d[1], h->d[2],
                                                 (const double *)R, ldr, (double *)W, ldw, nb, alpha, beta);
    else
        k_filter<float><<<blocks, 256, 0, st>>>(h->map.as<int32_t>(), h->loc.as<int32_t>(), h->npts, h->d[1], h->d[2],
                                                (const float *)R, ldr, (float *)W, ldw, nb, (float)alpha, (float)beta);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

}  // namespace rs

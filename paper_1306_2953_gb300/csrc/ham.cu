// Kohn-Sham Hamiltonian applied to a block of orbitals (Sec. V, Eq. 3).
//
// Two launches per block:
//  1. k_project: the Kleinman-Bylander projection integrals of Eq. (4),
//     c[A,q,s] = E[A,q] dV sum_{p in S_A} gamma_Aq(p) psi(p,s), PSPLIT CTAs
//     per (atom, state group), each a block-wide tree reduction over its share
//     of the sphere points added to the zeroed coefficients; stored
//     [atom][state][q] so that one 16-byte load gives a state's four.
//     FP32 blocks of 32-state groups take k_project_f32 (four states per lane
//     and four sphere entries per warp step, the atom split sized to fill the
//     GPU).
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
// FP32 blocks whose state count is a multiple of 32 take the persistent
// ring-buffer kernel of stencil_ring.cu for step 2 instead; k_stencil serves
// FP64 blocks, narrower state groups and layouts that kernel cannot copy.
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

// 1: FP32 blocks of 32 states go to the persistent ring-buffer kernel
// (stencil_ring.cu) when the block's layout allows 16-byte row copies.
#ifndef RS_STENCIL_RING
#define RS_STENCIL_RING 1
#endif

// Height (planes) of the z-slabs the ring kernel lays its columns out in
// before cutting them into per-CTA runs (the default: whole columns).
#ifndef RS_RING_SLAB
#define RS_RING_SLAB 4096
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

#ifndef RS_PROJ_CTAS
#define RS_PROJ_CTAS 5
#endif

// FP32 blocks of 32-state groups: lane l of a warp takes sphere entry
// l / 8 of the warp's four and the states 4 (l % 8) .. + 3 (one 16-byte
// load of the psi row), so a warp reads four psi rows per step; the grid is
// (atoms * split, state groups) with the split sized to fill the GPU.
constexpr int NTP4 = 256;

__global__ void __launch_bounds__(NTP4) k_project_f32(HamDev<float> d, const float *__restrict__ psi, int64_t ldp,
                                                     int nb, int split, float *__restrict__ cproj) {
    __shared__ float red[NTP4 / 32][8][16];
    const int A = blockIdx.x / split, part = blockIdx.x - A * split;
    const int sg0 = blockIdx.y * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 7;
    const int o = __ldg(d.sph_off + A), e = __ldg(d.sph_off + A + 1);
    const int per = (e - o + split - 1) / split;
    const int i0 = o + part * per, i1 = min(e, i0 + per);
    const float *ps = psi + sg0 + 4 * q;
    float acc[16];   // [projector][state]
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.f;
#pragma unroll 4
    for (int i = i0 + 4 * warp + (lane >> 3); i < i1; i += 4 * (NTP4 / 32)) {
        const int p = __ldg(d.sph_idx + i);
        const float4 v = __ldg(reinterpret_cast<const float4 *>(ps + (int64_t)p * ldp));
        const float4 g = __ldg(reinterpret_cast<const float4 *>(d.sph_gam) + i);
        const float gv[4] = {g.x, g.y, g.z, g.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int l = 0; l < 4; ++l)
#pragma unroll
            for (int st = 0; st < 4; ++st) acc[4 * l + st] = fmaf(gv[l], vv[st], acc[4 * l + st]);
    }
    // the four entries of a warp, then the warps
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 8);
        acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 16);
    }
    if (lane < 8) {
#pragma unroll
        for (int k = 0; k < 16; ++k) red[warp][q][k] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x < 128 && i0 < i1) {
        const int qq = threadIdx.x >> 4, k = threadIdx.x & 15, l = k >> 2, st = k & 3;
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < NTP4 / 32; ++w) t += red[w][qq][k];
        atomicAdd(cproj + ((int64_t)A * nb + sg0 + 4 * qq + st) * 4 + l, __ldg(d.E + 4 * A + l) * d.dV * t);
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

// ----------------------------------------------- face-neighbour filter ---
// W = alpha R + beta sum_{6 face neighbours} R (zero off the grid); one thread
// per (point, state), state fastest.
template <typename T>
__global__ void k_filter(const int32_t *__restrict__ map, const int32_t *__restrict__ loc, int64_t npts, int d1, int d2,
                         const T *__restrict__ R, int64_t ldr, T *__restrict__ W, int64_t ldw, int nb, T alpha,
                         T beta) {
    // block (nb, 256 / nb): threadIdx.x is the state, threadIdx.y the point
    const int s = threadIdx.x;
    const int64_t p = blockIdx.x * (int64_t)blockDim.y + threadIdx.y;
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
    int n_sm = 1;                  // SMs of the device (grid sizing)
    double w[5] = {0, 0, 0, 0, 0};
    DevBuf pinfo64, pinfo32, map, loc, V64, V32, cov_off, cov_atom, cov_gam64, cov_gam32, sph_off, sph_idx, sph_gam64, sph_gam32, E64, E32,
        cproj, dummy, scratch;
    std::map<std::pair<int, int>, WorkList *> work;
    RingPlan *ring = nullptr;      // tables of the ring-buffer FP32 kernel (nullptr: not usable)
    int kernel = RS_KERNEL_AUTO;   // rs_ham_select_kernel
    // optional per-launch timing (rs_ham_timing)
    bool timing = false;
    std::vector<cudaEvent_t> events;   // 3 per recorded call
    size_t n_recorded = 0;
    ~rs_ham() {
        ring_plan_destroy(ring);
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
    if (cudaDeviceGetAttribute(&H->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || H->n_sm < 1)
        return bail(fail(RS_ECUDA, "device query failed"));
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
#if RS_STENCIL_RING
    if ((rc = ring_plan_build(&H->ring, g, coff, catom, cg32, v32, (float)H->w[0], na, RS_RING_SLAB))) return bail(rc);
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
    RS_TRY(smem_optin((const void *)k_stencil<T, SG, TX, TY>, C::SMEM));
    const WorkList *wl = H->work.at({TX, TY});
    if (wl->count == 0) return RS_OK;
    dim3 grid((unsigned)wl->count, (unsigned)(nb / SG));
    k_stencil<T, SG, TX, TY><<<grid, C::NT, C::SMEM, st>>>(d, psi, ldp, hpsi, ldh, H->cproj.as<T>(), nb,
                                                            wl->buf.as<int4>());
    RS_LAUNCH_CHECK();
    return RS_OK;
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
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (nb % 32 == 0 && ldp % 4 == 0 && aligned16(psi)) {
                // one wave: at most RS_PROJ_CTAS CTAs of 256 threads per SM in all
                const int split = std::max(1, std::min(64, RS_PROJ_CTAS * H->n_sm / H->n_atoms));
                k_project_f32<<<dim3((unsigned)(H->n_atoms * split), (unsigned)(nb / 32)), NTP4, 0, st>>>(d, psi, ldp, nb,
                                                                                                        split, cp);
                done = true;
            }
        }
        if (!done) switch (sgp) {
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
                    if (H->kernel == RS_KERNEL_AUTO && ring_usable(H->ring, psi, ldp, nb)) {
                        float w[5];
                        for (int j = 0; j < 5; ++j) w[j] = (float)H->w[j];
                        rc = ring_launch(H->ring, psi, ldp, hpsi, ldh, H->cproj.as<float>(), nb, w, st);
                        break;
                    }
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
    // psi read once, hpsi written once, V and the point map, one copy of the
    // projector tables and the coefficients: the bytes of the fused launch
    // (the projection pass re-reads rows that stay in L2 and its own copy of
    // the tables, which are not counted again)
    int64_t b = 0;
    if (rs_ham_launch_bytes(h, nb, dtype, nullptr, &b) != RS_OK) return -1;
    return b;
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

__global__ void k_set_potential(const double *__restrict__ V, int64_t np, double *__restrict__ V64,
                                float *__restrict__ V32, int4 *__restrict__ p64, int4 *__restrict__ p32) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const double v = V[p];
        const float f = __double2float_rn(v);
        V64[p] = v;
        V32[p] = f;
        const long long bits = __double_as_longlong(v);
        int4 a = p64[p];
        a.z = (int)(bits & 0xffffffffll);
        a.w = (int)(bits >> 32);
        p64[p] = a;
        int4 b = p32[p];
        b.z = __float_as_int(f);
        p32[p] = b;
    }
}

extern "C" int rs_ham_set_potential(rs_ham *h, const double *V_dev, void *stream) {
    if (!h || !V_dev) return fail(RS_EINVAL, "rs_ham_set_potential: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    k_set_potential<<<(unsigned)std::min<int64_t>((h->npts + 255) / 256, 152 * 16), 256, 0, st>>>(
        V_dev, h->npts, h->V64.as<double>(), h->V32.as<float>(), h->pinfo64.as<int4>(), h->pinfo32.as<int4>());
    RS_LAUNCH_CHECK();
    return ring_set_potential(h->ring, h->V32.as<float>(), st);
}

extern "C" int rs_ham_select_kernel(rs_ham *h, int which) {
    if (!h || (which != RS_KERNEL_AUTO && which != RS_KERNEL_GENERIC)) return fail(RS_EINVAL, "rs_ham_select_kernel: bad argument");
    h->kernel = which;
    return RS_OK;
}

extern "C" int rs_ham_reset_status(rs_ham *h) {
    if (!h) return fail(RS_EINVAL, "rs_ham_reset_status: null handle");
    return ring_reset_status(h->ring);
}

extern "C" int rs_ham_set_wait_limit(rs_ham *h, int tests) {
    if (!h) return fail(RS_EINVAL, "rs_ham_set_wait_limit: null handle");
    ring_set_wait_limit(h->ring, tests);
    return RS_OK;
}

namespace rs {
int *ham_status_word(rs_ham *h) { return ring_status_word(h->ring); }
}  // namespace rs

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
    const dim3 blk((unsigned)nb, (unsigned)std::max(1, 256 / nb));
    const unsigned blocks = (unsigned)((h->npts + blk.y - 1) / blk.y);
    const double beta = (1.0 - alpha) / 6.0;
    if (dtype == RS_F64)
        k_filter<double><<<blocks, blk, 0, st>>>(h->map.as<int32_t>(), h->loc.as<int32_t>(), h->npts, h->d[1], h->d[2],
                                                 (const double *)R, ldr, (double *)W, ldw, nb, alpha, beta);
    else
        k_filter<float><<<blocks, blk, 0, st>>>(h->map.as<int32_t>(), h->loc.as<int32_t>(), h->npts, h->d[1], h->d[2],
                                                (const float *)R, ldr, (float *)W, ldw, nb, (float)alpha, (float)beta);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

}  // namespace rs

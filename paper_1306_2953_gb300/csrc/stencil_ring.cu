// Fused Kohn-Sham H psi for FP32 blocks of 32 states (Sec. V, Eq. 3): the
// 25-point star kinetic stencil (Sec. V.A), the local potential (Sec. V.B)
// and the nonlocal gather of Eq. (4), one persistent CTA per SM.
//
// Work.  The point map is cut into 8 x 8 columns (map axes 1 and 2) and each
// column into z-slabs along the march axis 0; a unit is (column, slab).  The
// host deals the units of every slab to the CTAs, largest first onto the
// least loaded CTA, and each CTA takes its units slab by slab: at any moment
// the CTAs march neighbouring columns of the same slab, so the halo rows
// they share are re-read from L2 rather than HBM.  blockIdx.y is the state
// group (32 states) of the block.
//
// Ring.  A CTA keeps RING planes of its column in shared memory.  A slot
// holds one plane of the 16 x 16 window (the 8 x 8 tile and its 4-point
// star halo in both in-plane axes), 128 bytes (32 FP32 states) per lattice
// position, plus the plane's record: per tile point its potential, point
// index and nonlocal entries (projector values and atom).  Every thread
// copies its share of plane it + AHEAD while plane it is computed: three
// 16-byte pieces of point rows (eight threads per row; absent points are
// zero-filled) and part of the record, all counted on the slot's "full"
// mbarrier through cp.async.mbarrier.arrive.  A slot is refilled once every
// warp has released it ("empty" mbarrier).  Points are stored brick by brick
// (Sec. V.A), so one 32-bit descriptor (first point, presence mask) gives
// the four points of a brick row.
//
// Compute.  Warp w owns the 2 x 2 patch of tile points at (2 (w / 4),
// 2 (w % 4)); lane s is state s.  Pairs of points along axis 2 share packed
// FP32x2 instructions.  The march accumulates forward: the values of plane z
// add w_|j| psi(z) to the outputs of planes z + j (j = -4..4, nine
// accumulators per point in registers, addressed by z mod 9 through
// unrolling), and the in-plane star, the potential and the nonlocal sum to
// plane z's own output, so a slot is read in one step only and output
// z - 4 is complete, and written once, at step z.  The four planes on either
// side of a slab contribute only their z-terms (tile rows only, no record).
//
// Every mbarrier wait is bounded; on a timeout the kernel sets its status
// word and leaves the march.
#include <algorithm>
#include <cstring>
#include <new>

#include "device.h"
#include "stencil_ring.h"

#ifndef RS_RING_SLOTS
#define RS_RING_SLOTS 4
#endif
#ifndef RS_RING_AHEAD
#define RS_RING_AHEAD (RS_RING_SLOTS - 2)
#endif

namespace rs {

namespace {

constexpr int TT = 8;                      // tile edge (lattice points)
constexpr int WIN = TT + 8;                // window edge
constexpr int SG = 32;                     // states per CTA
constexpr int ROWB = SG * 4;               // bytes per point row
constexpr int SLOT_PSI = WIN * WIN * ROWB;
constexpr int NG = 48;                     // brick rows of four positions per window plane
constexpr int NG_CORE = 16;                // brick rows of the tile itself
constexpr int NW = 16;                     // warps: one 2 x 2 patch each
constexpr int NT = NW * 32;
constexpr int RING = RS_RING_SLOTS;
constexpr int AHEAD = RS_RING_AHEAD;       // planes in flight ahead of the one computed
static_assert(AHEAD >= 1 && AHEAD < RING, "copy distance must leave a slot to compute on");
constexpr int NPOS = TT * TT;
constexpr int REC_HDR = 16;                // record header: entries count
constexpr int META_BYTES = NPOS * 16;
constexpr int MAX_REC = 40 * 1024;         // record slot budget (bytes)
constexpr size_t MAX_SMEM = 227 * 1024;    // dynamic shared memory per CTA
constexpr int MAX_SLAB = 128;              // planes per z-slab of a unit (at most)
constexpr int MAX_UNITS = 64;              // units per CTA (shared-memory table)
constexpr int SUSPEND_NS = 20000;           // suspension limit of one barrier test
constexpr int SPIN = 100000;               // barrier tests before a wait gives up

// Window position (row yw, first column xw) of brick row g: 0..15 the tile,
// 16..31 the axis-2 halo beside it, 32..47 the axis-1 halo above and below.
__host__ __device__ __forceinline__ void group_pos(int g, int &yw, int &xw) {
    if (g < 16) {
        yw = 4 + (g >> 1);
        xw = 4 + 4 * (g & 1);
    } else if (g < 32) {
        const int h = g - 16;
        yw = 4 + (h >> 1);
        xw = (h & 1) ? 12 : 0;
    } else {
        const int h = g - 32, r = h >> 1;
        yw = r < 4 ? r : r + 8;
        xw = 4 + 4 * (h & 1);
    }
}

// A unit as the kernel walks it: planes zm0..zm1 (the slab's output planes
// zo0..zo1-1 and up to four on either side), record / descriptor index of
// plane z = pz + z.
struct UnitDev {
    int zm0, zm1, zo0, zo1, pz, pad0, pad1, pad2;
};

struct Args {
    const UnitDev *units;   // per CTA, concatenated
    const int2 *cta;        // [CTA]: first unit, unit count
    const uint32_t *desc;   // [plane][48]: first point | presence mask << 28
    const uint2 *recs;      // [plane]: {offset / 16, bytes}
    const unsigned char *rec;
    const float *psi;       // [npts][ldp]
    int64_t ldp;
    const float *cproj;     // [atom][nb][4]
    float *hpsi;
    int64_t ldh;
    int nb, n_atoms, rec_slot;
    float w[5];
    int *status;
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(b)) : "memory");
}
// One bounded test of the phase: the thread is suspended until the phase
// completes or SUSPEND_NS nanoseconds have passed, so a waiting warp does not
// take issue slots from the warps that compute.
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "n"(SUSPEND_NS)
        : "memory");
    return ok != 0;
}
// at most SPIN tests (about SPIN * SUSPEND_NS, two seconds, in all)
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity) {
    for (int i = 0; i < SPIN; ++i)
        if (bar_try(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
// arrive on the mbarrier once every cp.async this thread issued so far has landed
__device__ __forceinline__ void cp_async_arrive(uint64_t *b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }

struct Lane {
    float2 W1, W2, W3, W4;
    float w0;
    int lx, ly, s;
};

// Window position index of tile point (y, x) shifted by (dy, dx).
__device__ __forceinline__ int wpos(int y, int x) { return (y + 4) * WIN + x + 4; }

// One march step over plane z (R = z mod 9).  A[k][dy] holds the outputs of
// the patch row dy (x: point dx = 0, y: dx = 1) for plane z' = k mod 9.
template <int R>
__device__ __forceinline__ void march(float2 (&A)[9][2], const float *__restrict__ P, const unsigned char *rs,
                                      int *rowring, bool full, const float *__restrict__ cpl, int nb4, const Lane &c) {
    float2 u[2];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
        u[dy] = make_float2(P[wpos(c.ly + dy, c.lx) * SG + c.s], P[wpos(c.ly + dy, c.lx + 1) * SG + c.s]);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        const float2 v = u[dy];
        A[(R + 1) % 9][dy] = fma2(c.W1, v, A[(R + 1) % 9][dy]);
        A[(R + 8) % 9][dy] = fma2(c.W1, v, A[(R + 8) % 9][dy]);
        A[(R + 2) % 9][dy] = fma2(c.W2, v, A[(R + 2) % 9][dy]);
        A[(R + 7) % 9][dy] = fma2(c.W2, v, A[(R + 7) % 9][dy]);
        A[(R + 3) % 9][dy] = fma2(c.W3, v, A[(R + 3) % 9][dy]);
        A[(R + 6) % 9][dy] = fma2(c.W3, v, A[(R + 6) % 9][dy]);
        A[(R + 4) % 9][dy] = fma2(c.W4, v, A[(R + 4) % 9][dy]);
        A[(R + 5) % 9][dy] = fma2(c.W4, v, A[(R + 5) % 9][dy]);
    }
    if (!full) return;
    const int E = *reinterpret_cast<const int *>(rs);
    const int4 *meta = reinterpret_cast<const int4 *>(rs + REC_HDR);
    const float4 *gam = reinterpret_cast<const float4 *>(rs + REC_HDR + META_BYTES);
    const int *atom = reinterpret_cast<const int *>(rs + REC_HDR + META_BYTES + 16 * E);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        const int pos = (c.ly + dy) * TT + c.lx;
        const int4 m0 = meta[pos], m1 = meta[pos + 1];
        if (c.s == 0) {
            rowring[R * NPOS + pos] = m0.y;
            rowring[R * NPOS + pos + 1] = m1.y;
        }
        // centre of the star and the potential
        float2 a = fma2(make_float2(c.w0 + __int_as_float(m0.x), c.w0 + __int_as_float(m1.x)), u[dy], A[R][dy]);
        // nonlocal gather over the atoms whose spheres cover each point: the
        // two points' entry lists are walked side by side (independent load
        // and multiply chains), each projection a two-level sum
        const int n0 = m0.w, n1 = m1.w, nmax = max(n0, n1);
        for (int k = 0; k < nmax; ++k) {
            const int e0 = m0.z + min(k, n0 - 1), e1 = m1.z + min(k, n1 - 1);
            const float4 g0 = gam[max(e0, 0)], g1 = gam[max(e1, 0)];
            const int a0 = atom[max(e0, 0)], a1 = atom[max(e1, 0)];
            const float4 c0 = *reinterpret_cast<const float4 *>(cpl + a0 * nb4);
            const float4 c1 = *reinterpret_cast<const float4 *>(cpl + a1 * nb4);
            const float p0 = (g0.x * c0.x + g0.y * c0.y) + (g0.z * c0.z + g0.w * c0.w);
            const float p1 = (g1.x * c1.x + g1.y * c1.y) + (g1.z * c1.z + g1.w * c1.w);
            if (k < n0) a.x += p0;
            if (k < n1) a.y += p1;
        }
        // axis-2 neighbours: the window row of the patch row
        float v[10];
#pragma unroll
        for (int k = 0; k < 10; ++k)
            if (k != 4 && k != 5) v[k] = P[wpos(c.ly + dy, c.lx + k - 4) * SG + c.s];
        v[4] = u[dy].x;
        v[5] = u[dy].y;
        // two short independent chains (j = 1, 3 and j = 2, 4) instead of one
        float2 x13 = c.W1 * add2(make_float2(v[5], v[6]), make_float2(v[3], v[4]));
        float2 x24 = c.W2 * add2(make_float2(v[6], v[7]), make_float2(v[2], v[3]));
        x13 = fma2(c.W3, add2(make_float2(v[7], v[8]), make_float2(v[1], v[2])), x13);
        x24 = fma2(c.W4, add2(make_float2(v[8], v[9]), make_float2(v[0], v[1])), x24);
        A[R][dy] = add2(a, add2(x13, x24));
    }
    // axis-1 neighbours: the window columns of the patch, both columns paired
    float2 col[10];
#pragma unroll
    for (int k = 0; k < 10; ++k)
        if (k != 4 && k != 5)
            col[k] = make_float2(P[wpos(c.ly + k - 4, c.lx) * SG + c.s], P[wpos(c.ly + k - 4, c.lx + 1) * SG + c.s]);
    col[4] = u[0];
    col[5] = u[1];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        float2 y13 = c.W1 * add2(col[5 + dy], col[3 + dy]);
        float2 y24 = c.W2 * add2(col[6 + dy], col[2 + dy]);
        y13 = fma2(c.W3, add2(col[7 + dy], col[1 + dy]), y13);
        y24 = fma2(c.W4, add2(col[8 + dy], col[0 + dy]), y24);
        A[R][dy] = add2(A[R][dy], add2(y13, y24));
    }
}

// Writes the finished output of plane o (R = o mod 9) when `store`, and
// clears its accumulators for plane o + 9.
template <int R>
__device__ __forceinline__ void emit(float2 (&A)[9][2], const int *rowring, float *hp, int64_t ldh, bool store,
                                     const Lane &c) {
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        if (store) {
            const int pos = (c.ly + dy) * TT + c.lx;
            const int r0 = rowring[R * NPOS + pos], r1 = rowring[R * NPOS + pos + 1];
            if (r0 >= 0) hp[(int64_t)r0 * ldh] = A[R][dy].x;
            if (r1 >= 0) hp[(int64_t)r1 * ldh] = A[R][dy].y;
        }
        A[R][dy] = make_float2(0.f, 0.f);
    }
}

template <int R>
__device__ __forceinline__ void step(float2 (&A)[9][2], const float *P, const unsigned char *rs, int *rowring,
                                     uint64_t *ebar, bool full, const float *cpl, int nb4, float *hp, int64_t ldh,
                                     bool store, const Lane &c) {
    march<R>(A, P, rs, rowring, full, cpl, nb4, c);
    __syncwarp();
    if (c.s == 0) bar_arrive(ebar);   // the slot is no longer read by this warp
    emit<(R + 5) % 9>(A, rowring, hp, ldh, store, c);
}

__device__ __forceinline__ void emit_any(int r, float2 (&A)[9][2], const int *rowring, float *hp, int64_t ldh,
                                         const Lane &c) {
    switch (r) {
        case 0: emit<0>(A, rowring, hp, ldh, true, c); break;
        case 1: emit<1>(A, rowring, hp, ldh, true, c); break;
        case 2: emit<2>(A, rowring, hp, ldh, true, c); break;
        case 3: emit<3>(A, rowring, hp, ldh, true, c); break;
        case 4: emit<4>(A, rowring, hp, ldh, true, c); break;
        case 5: emit<5>(A, rowring, hp, ldh, true, c); break;
        case 6: emit<6>(A, rowring, hp, ldh, true, c); break;
        case 7: emit<7>(A, rowring, hp, ldh, true, c); break;
        default: emit<8>(A, rowring, hp, ldh, true, c); break;
    }
}

// Position of the CTA in its unit list: unit k (a copy in U), plane z.
struct Cursor {
    int k, z;
    UnitDev U;
};

// CPS: the projection coefficients of the CTA's state group are staged in
// shared memory (when they fit), so the nonlocal gather reads no global memory.
template <bool CPS>
__global__ void __launch_bounds__(NT, 1) k_hpsi_ring(Args a) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *psi_ring = base;                                         // [RING] windows
    unsigned char *rec_ring = base + (size_t)RING * SLOT_PSI;              // [RING] records
    UnitDev *ut = reinterpret_cast<UnitDev *>(rec_ring + (size_t)RING * a.rec_slot);   // [MAX_UNITS]
    int *rowring = reinterpret_cast<int *>(ut + MAX_UNITS);                 // [9][NPOS] output rows
    int *wrow = rowring + 9 * NPOS;                                         // [NG * 4] window position of each row
    float *cps = reinterpret_cast<float *>(wrow + NG * 4);                  // [atom][32 states][4] when CPS
    __shared__ uint64_t fullb[RING], emptyb[RING];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = blockIdx.y;
    const int2 mine = a.cta[blockIdx.x];
    const int nu = min(mine.y, MAX_UNITS);
    if (tid == 0) {
        for (int i = 0; i < RING; ++i) {
            bar_init(&fullb[i], NT);    // every thread's copy completions
            bar_init(&emptyb[i], NW);   // every warp's release
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int k = tid; k < nu; k += NT) ut[k] = a.units[mine.x + k];
    for (int r = tid; r < NG * 4; r += NT) {
        int yw, xw;
        group_pos(r >> 2, yw, xw);
        wrow[r] = yw * WIN + xw + (r & 3);
    }
    if (CPS) {
        const float4 *src = reinterpret_cast<const float4 *>(a.cproj);
        float4 *dst = reinterpret_cast<float4 *>(cps);
        for (int e = tid; e < a.n_atoms * SG; e += NT) {
            const int at = e / SG, st = e - at * SG;
            dst[e] = __ldg(src + (int64_t)at * a.nb + grp * SG + st);
        }
    }
    __syncthreads();
    if (nu == 0) return;

    // ---- copies: plane of cursor q into slot j % RING.  The plane's
    // descriptors (the three window rows this thread copies) and record
    // address are loaded one plane ahead.
    bool ok = true;
    const float *src0 = a.psi + grp * SG + 4 * (tid & 7);
    // this thread copies bytes 16 (tid % 8) .. of window rows tid / 8 + 64 k:
    // their slot offsets and brick-row bit are fixed
    int doff[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) doff[k] = wrow[(tid >> 3) + (NT / 8) * k] * ROWB + 16 * (tid & 7);
    const uint32_t rbit = 1u << ((tid >> 3) & 3);
    struct Pre {
        uint32_t d[3];
        uint2 rc;
        bool full;
    };
    auto prefetch = [&](const Cursor &q, Pre &f) {
        const UnitDev &U = q.U;
        f.full = q.z >= U.zo0 && q.z < U.zo1;
        const int64_t pt = (int64_t)U.pz + q.z;
        const int nrow = f.full ? NG * 4 : NG_CORE * 4;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = (tid >> 3) + (NT / 8) * k;
            f.d[k] = r < nrow ? __ldg(a.desc + pt * NG + (r >> 2)) : 0u;
        }
        f.rc = f.full ? __ldg(a.recs + pt) : make_uint2(0u, 0u);
    };
    auto issue = [&](int j, const Pre &f) {
        const int slot = j % RING;
        if (!__all_sync(0xffffffffu, j < RING || bar_wait(&emptyb[slot], ((j / RING) - 1) & 1))) {
            ok = false;
            return;
        }
        unsigned char *dst = psi_ring + (size_t)slot * SLOT_PSI;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k > 0 && !f.full) break;   // edge planes: the tile rows only (r < 64)
            const uint32_t d = f.d[k];
            const uint32_t mask = d >> 28;
            const bool has = (mask & rbit) != 0;
            const int pnt = (int)(d & 0x0fffffffu) + __popc(mask & (rbit - 1u));
            cp_async16(dst + doff[k], has ? src0 + (int64_t)pnt * a.ldp : src0, has);
        }
        if (f.full) {
            const unsigned char *rsrc = a.rec + (size_t)f.rc.x * 16;
            unsigned char *rdst = rec_ring + (size_t)slot * a.rec_slot;
            for (int o = tid * 16; o < (int)f.rc.y; o += NT * 16) cp_async16(rdst + o, rsrc + o, true);
        }
        cp_async_arrive(&fullb[slot]);
    };
    auto advance = [&](Cursor &q) {
        if (++q.z > q.U.zm1) {
            ++q.k;
            if (q.k < nu) {
                q.U = ut[q.k];
                q.z = q.U.zm0;
            }
        }
    };

    Lane c;
    c.w0 = a.w[0];
    c.W1 = f2(a.w[1]);
    c.W2 = f2(a.w[2]);
    c.W3 = f2(a.w[3]);
    c.W4 = f2(a.w[4]);
    c.s = lane;
    c.lx = 2 * (warp & 3);
    c.ly = 2 * (warp >> 2);
    const int nb4 = CPS ? SG * 4 : a.nb * 4;
    const float *cpl = CPS ? cps + lane * 4 : a.cproj + (int64_t)(grp * SG + lane) * 4;
    float *hp = a.hpsi + grp * SG + lane;
    float2 A[9][2];
#pragma unroll
    for (int k = 0; k < 9; ++k) A[k][0] = A[k][1] = make_float2(0.f, 0.f);

    Cursor qi{0, ut[0].zm0, ut[0]}, qc{0, ut[0].zm0, ut[0]};
    Pre pre;
    prefetch(qi, pre);
    int j = 0;   // planes issued
    for (; j < AHEAD && qi.k < nu && ok; ++j) {
        issue(j, pre);
        advance(qi);
        if (qi.k < nu) prefetch(qi, pre);
    }
    for (int it = 0; qc.k < nu && ok; ++it) {
        if (qi.k < nu) {
            issue(j++, pre);
            advance(qi);
            if (!ok) break;
            if (qi.k < nu) prefetch(qi, pre);
        }
        const int slot = it % RING;
        if (!__all_sync(0xffffffffu, bar_wait(&fullb[slot], (it / RING) & 1))) {
            ok = false;
            break;
        }
        const UnitDev &U = qc.U;
        const int z = qc.z;
        if (z == U.zm0) {
#pragma unroll
            for (int k = 0; k < 9; ++k) A[k][0] = A[k][1] = make_float2(0.f, 0.f);
        }
        const bool full = z >= U.zo0 && z < U.zo1;
        const float *P = reinterpret_cast<const float *>(psi_ring + (size_t)slot * SLOT_PSI);
        const unsigned char *rs = rec_ring + (size_t)slot * a.rec_slot;
        uint64_t *eb = &emptyb[slot];
        const bool st = z - 4 >= U.zo0 && z - 4 < U.zo1;
        switch (z % 9) {
            case 0: step<0>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            case 1: step<1>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            case 2: step<2>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            case 3: step<3>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            case 4: step<4>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            case 5: step<5>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            case 6: step<6>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            case 7: step<7>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
            default: step<8>(A, P, rs, rowring, eb, full, cpl, nb4, hp, a.ldh, st, c); break;
        }
        // last plane of the column inside the unit: planes beyond it are
        // empty, so the outputs still open are complete
        if (z == U.zm1 && z < U.zo1 + 3) {
            __syncwarp();
            for (int o = z - 3; o <= z; ++o)
                if (o >= U.zo0 && o < U.zo1) emit_any(o % 9, A, rowring, hp, a.ldh, c);
        }
        advance(qc);
    }
    if (!ok && lane == 0) atomicExch(a.status, 1);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace

struct RingPlan {
    DevBuf units, cta, desc, recs, rec, status;
    int n_cta = 0, rec_slot = 0, n_atoms = 0;
    int64_t npts = 0;
    size_t smem = 0;          // without staged coefficients
    size_t smem_cps = 0;      // with the coefficients of one state group staged
    int smem_set[2] = {0, 0};
};

void ring_plan_destroy(RingPlan *p) { delete p; }

int ring_plan_build(RingPlan **out, const rs_grid *g, const std::vector<int32_t> &coff, const std::vector<int32_t> &catom,
                    const std::vector<float> &cg32, const std::vector<float> &v32, int n_atoms, int slab) {
    *out = nullptr;
    if (g->npts >= (1 << 28) || slab < 1 || slab > MAX_SLAB) return RS_OK;
    const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
    auto at = [&](int a0, int a1, int a2) -> int32_t {
        if (a0 < 0 || a1 < 0 || a2 < 0 || a0 >= d0 || a1 >= d1 || a2 >= d2) return -1;
        return g->map[((size_t)a0 * d1 + a1) * d2 + a2];
    };
    const int n1 = (d1 + TT - 1) / TT, n2 = (d2 + TT - 1) / TT;
    struct Col {
        int zmin, zmax;
        int64_t p0;   // record / descriptor index of plane zmin
    };
    std::vector<Col> cols;
    std::vector<uint32_t> desc;
    std::vector<uint2> recs;
    std::vector<int32_t> blob;   // 4-byte words; records start on 16-byte boundaries
    int max_rec = 0;
    int64_t nplanes = 0;
    try {
        for (int t1 = 0; t1 < n1; ++t1)
            for (int t2 = 0; t2 < n2; ++t2) {
                const int b1 = t1 * TT, b2 = t2 * TT;
                int zmin = d0, zmax = -1;
                for (int a0 = 0; a0 < d0; ++a0)
                    for (int iy = 0; iy < TT; ++iy)
                        for (int ix = 0; ix < TT; ++ix)
                            if (at(a0, b1 + iy, b2 + ix) >= 0) {
                                zmin = std::min(zmin, a0);
                                zmax = std::max(zmax, a0);
                            }
                if (zmax < 0) continue;
                cols.push_back({zmin, zmax, nplanes});
                for (int z = zmin; z <= zmax; ++z) {
                    for (int gi = 0; gi < NG; ++gi) {
                        int yw, xw;
                        group_pos(gi, yw, xw);
                        uint32_t mask = 0;
                        int32_t first = -1, prev = -1;
                        for (int i = 0; i < 4; ++i) {
                            const int32_t m = at(z, b1 + yw - 4, b2 + xw - 4 + i);
                            if (m < 0) continue;
                            if (first < 0) first = m;
                            else if (m != prev + 1) return fail(RS_EINVAL, "stencil plan: brick row not consecutive");
                            prev = m;
                            mask |= 1u << i;
                        }
                        desc.push_back((mask << 28) | (uint32_t)(first < 0 ? 0 : first));
                    }
                    // record: {entries}, meta[64] {V bits, point, first entry, entries},
                    // projector values [entries][4], atoms [entries] (padded)
                    const size_t off = blob.size();
                    int4 meta[NPOS];
                    std::vector<float> gm;
                    std::vector<int32_t> am;
                    for (int iy = 0; iy < TT; ++iy)
                        for (int ix = 0; ix < TT; ++ix) {
                            const int32_t m = at(z, b1 + iy, b2 + ix);
                            if (m < 0) {
                                meta[iy * TT + ix] = make_int4(0, -1, 0, 0);
                                continue;
                            }
                            int32_t vb;
                            memcpy(&vb, &v32[m], 4);
                            const int e0 = coff[m], e1 = coff[m + 1];
                            meta[iy * TT + ix] = make_int4(vb, m, (int)am.size(), e1 - e0);
                            for (int e = e0; e < e1; ++e) {
                                for (int q = 0; q < 4; ++q) gm.push_back(cg32[(size_t)e * 4 + q]);
                                am.push_back(catom[e]);
                            }
                        }
                    const int E = (int)am.size();
                    while (am.size() % 4) am.push_back(0);
                    blob.push_back(E);
                    blob.push_back(0);
                    blob.push_back(0);
                    blob.push_back(0);
                    for (int i = 0; i < NPOS; ++i) {
                        blob.push_back(meta[i].x);
                        blob.push_back(meta[i].y);
                        blob.push_back(meta[i].z);
                        blob.push_back(meta[i].w);
                    }
                    for (float f : gm) {
                        int32_t b;
                        memcpy(&b, &f, 4);
                        blob.push_back(b);
                    }
                    blob.insert(blob.end(), am.begin(), am.end());
                    const int bytes = (int)((blob.size() - off) * 4);
                    max_rec = std::max(max_rec, bytes);
                    if (off / 4 > UINT32_MAX) return RS_OK;
                    recs.push_back(make_uint2((uint32_t)(off / 4), (uint32_t)bytes));
                    ++nplanes;
                }
            }
        if (cols.empty() || max_rec > MAX_REC) return RS_OK;
        int dev = 0, n_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return fail(RS_ECUDA, "device query failed");
        // units slab by slab; within a slab, largest unit first onto the least
        // loaded CTA (cost: planes marched, edge planes at a quarter)
        const int G = std::max(1, n_sm);
        std::vector<std::vector<UnitDev>> per(G);
        std::vector<double> load(G, 0.0);
        const int nslab = (d0 + slab - 1) / slab;
        for (int s = 0; s < nslab; ++s) {
            std::vector<std::pair<double, UnitDev>> us;
            for (const Col &cl : cols) {
                const int zo0 = std::max(cl.zmin, s * slab), zo1 = std::min(cl.zmax + 1, (s + 1) * slab);
                if (zo0 >= zo1) continue;
                UnitDev u{};
                u.zo0 = zo0;
                u.zo1 = zo1;
                u.zm0 = std::max(cl.zmin, zo0 - 4);
                u.zm1 = std::min(cl.zmax, zo1 + 3);
                const int64_t pz = cl.p0 - cl.zmin;
                if (pz < INT32_MIN || pz > INT32_MAX) return RS_OK;
                u.pz = (int)pz;
                const double cost = (zo1 - zo0) + 0.25 * ((u.zm1 - u.zm0 + 1) - (zo1 - zo0));
                us.push_back({cost, u});
            }
            std::stable_sort(us.begin(), us.end(), [](const std::pair<double, UnitDev> &x, const std::pair<double, UnitDev> &y) {
                return x.first > y.first;
            });
            for (const auto &cu : us) {
                const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                per[k].push_back(cu.second);
                load[k] += cu.first;
            }
        }
        std::vector<UnitDev> flat;
        std::vector<int2> cta(G);
        for (int k = 0; k < G; ++k) {
            if (per[k].size() > (size_t)MAX_UNITS) return RS_OK;
            cta[k] = make_int2((int)flat.size(), (int)per[k].size());
            flat.insert(flat.end(), per[k].begin(), per[k].end());
        }
        RingPlan *P = new (std::nothrow) RingPlan;
        if (!P) return fail(RS_ENOMEM, "host allocation failed");
        auto bail = [&](int rc) {
            delete P;
            return rc;
        };
        int rc;
        if ((rc = P->units.upload(flat.data(), flat.size() * sizeof(UnitDev))) ||
            (rc = P->cta.upload(cta.data(), cta.size() * sizeof(int2))) ||
            (rc = P->desc.upload(desc.data(), desc.size() * sizeof(uint32_t))) ||
            (rc = P->recs.upload(recs.data(), recs.size() * sizeof(uint2))) ||
            (rc = P->rec.upload(blob.data(), blob.size() * sizeof(int32_t))) || (rc = P->status.alloc(sizeof(int))))
            return bail(rc);
        if (cudaMemset(P->status.p, 0, sizeof(int)) != cudaSuccess) return bail(fail(RS_ECUDA, "cudaMemset failed"));
        P->n_cta = G;
        P->rec_slot = (max_rec + 127) & ~127;
        P->npts = g->npts;
        P->n_atoms = n_atoms;
        P->smem = 1024 + (size_t)RING * (SLOT_PSI + P->rec_slot) + MAX_UNITS * sizeof(UnitDev) + 9 * NPOS * sizeof(int) +
                  NG * 4 * sizeof(int);
        P->smem_cps = P->smem + (size_t)n_atoms * SG * 4 * sizeof(float);
        if (P->smem > MAX_SMEM) return bail(RS_OK);
        *out = P;
    } catch (const std::bad_alloc &) {
        return fail(RS_ENOMEM, "host allocation failed");
    }
    return RS_OK;
}

bool ring_usable(const RingPlan *p, const float *psi, int64_t ldp, int nb) {
    return p && nb % SG == 0 && ldp % 4 == 0 && aligned16(psi);
}

int ring_launch(RingPlan *p, const float *psi, int64_t ldp, float *hpsi, int64_t ldh, const float *cproj, int nb,
                const float w[5], cudaStream_t st) {
    Args a;
    a.units = p->units.as<UnitDev>();
    a.cta = p->cta.as<int2>();
    a.desc = p->desc.as<uint32_t>();
    a.recs = p->recs.as<uint2>();
    a.rec = p->rec.as<unsigned char>();
    a.psi = psi;
    a.ldp = ldp;
    a.cproj = cproj;
    a.hpsi = hpsi;
    a.ldh = ldh;
    a.nb = nb;
    a.n_atoms = p->n_atoms;
    a.rec_slot = p->rec_slot;
    for (int j = 0; j < 5; ++j) a.w[j] = w[j];
    a.status = p->status.as<int>();
    const dim3 grid((unsigned)p->n_cta, (unsigned)(nb / SG));
    if (p->n_atoms > 0 && p->smem_cps <= MAX_SMEM) {
        if (p->smem_set[1] < (int)p->smem_cps) {
            RS_CUDA(cudaFuncSetAttribute(k_hpsi_ring<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_cps));
            p->smem_set[1] = (int)p->smem_cps;
        }
        k_hpsi_ring<true><<<grid, NT, p->smem_cps, st>>>(a);
    } else {
        if (p->smem_set[0] < (int)p->smem) {
            RS_CUDA(cudaFuncSetAttribute(k_hpsi_ring<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem));
            p->smem_set[0] = (int)p->smem;
        }
        k_hpsi_ring<false><<<grid, NT, p->smem, st>>>(a);
    }
    RS_LAUNCH_CHECK();
    return RS_OK;
}

int ring_status(const RingPlan *p, int *flag) {
    *flag = 0;
    if (!p) return RS_OK;
    RS_CUDA(cudaMemcpy(flag, p->status.as<int>(), sizeof(int), cudaMemcpyDeviceToHost));
    return RS_OK;
}

}  // namespace rs

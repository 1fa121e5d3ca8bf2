// Fused Kohn-Sham H psi for FP32 blocks of 32 states (Sec. V, Eq. 3): the
// 25-point star kinetic stencil (Sec. V.A), the local potential (Sec. V.B)
// and the nonlocal gather of Eq. (4), one persistent CTA per SM.
//
// Work.  The point map is cut into 16 x 8 tiles (16 along map axis 2, 8
// along axis 1); a tile column is marched along axis 0.  The host lays the
// columns out slab by slab (z-slabs of a given height; the default is one
// slab, whole columns) in raster order and cuts that sequence into one
// contiguous run per CTA of equal modelled cost, splitting a column at a
// plane where a run ends; a unit is such a piece of a column.  blockIdx.y is
// the state group (32 states) of the block.
//
// Ring.  A CTA keeps RING planes (4, or 3 when 4 do not fit in shared
// memory) of its column in shared memory.  A slot holds the 320 window
// positions one plane of the star reads (the tile, 4 rows above and below
// it, 4 columns left and right of it; the window's corners are not stored),
// 128 bytes (32 FP32 states) per position, plus the plane's record: the
// potential and the point index of every tile point and, per 4 x 4 patch,
// the projector values of each atom whose sphere meets the patch (zero at
// the patch points outside the sphere).  Every thread copies its share of
// plane it + 2 while plane it is computed: one 16-byte piece of ten point
// rows (a warp copies a 4-point brick row per instruction; absent points are
// zero-filled) and part of the record, all counted on the slot's "full"
// mbarrier through cp.async.mbarrier.arrive.  A slot is refilled once every
// warp has released it ("empty" mbarrier).  Points are stored brick by brick
// (Sec. V.A), so one 32-bit descriptor (first point, presence mask) gives
// the four points of a brick row; the descriptors are loaded three planes
// ahead of their copy.  The projection coefficients of the atoms a CTA's
// records name are staged in shared memory once per launch (the records
// carry the CTA-local atom numbers).
//
// Compute.  Warp w owns the 4 x 4 patch of tile points at rows 4 (w / 4),
// columns 4 (w % 4); half-warp h takes the patch's rows 2h and 2h + 1 and
// lane l of the half the states 2l and 2l + 1, so every value is a pair of
// states and every multiply-add a packed FP32x2 instruction.  The march
// accumulates forward: the values of plane z add w_|j| psi(z) to the outputs
// of planes z + j (j = -4..4), and the in-plane star, the potential and the
// nonlocal sum to plane z's own output, so a slot is read in one step only.
// Eight accumulators per point hold the outputs z - 4 .. z + 3 (slot z mod 8,
// addressed through unrolling): at step z output z - 4 is complete and
// written, and its slot takes output z + 4.  The four planes on either side
// of a unit contribute only their z-terms (tile rows only, no record).
//
// Every mbarrier wait is bounded; on a timeout the kernel sets its status
// word and leaves the march.  Built with RS_BOUNDS_CHECK=1 (a debugging
// build standing in for a memory checker), every point index the kernel
// copies from or stores to is tested against the point count first; an index
// out of range is skipped and sets bit 2 of the status word.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>

#include "device.h"
#include "stencil_ring.h"

#ifndef RS_BOUNDS_CHECK
#define RS_BOUNDS_CHECK 0
#endif

namespace rs {

namespace {

constexpr int TX = 16;                     // tile extent along map axis 2
constexpr int TY = 8;                      // tile extent along map axis 1
constexpr int SG = 32;                     // states per CTA
constexpr int ROWB = SG * 4;               // bytes per point row
constexpr int NSLOT = 320;                 // stored window positions
constexpr int SLOT_PSI = NSLOT * ROWB;
constexpr int NG = 80;                     // brick rows (four positions) per window plane
constexpr int NW = 8;                      // warps: one 4 x 4 patch each
constexpr int NT = NW * 32;
constexpr int CPW = NG / NW;               // brick rows copied per warp and plane

// host load balance: march cost of an edge plane and of one atom block of a
// plane's heaviest patch, in full planes (fitted to per-CTA clock counts)
constexpr double EDGE_COST = 0.38;
constexpr double NL_COST = 0.09;
constexpr int AHEAD = 2;                   // planes in flight ahead of the one computed
constexpr int MAX_RING = 4;                // slots per CTA (4, or 3 when 4 do not fit)
constexpr int NPOS = TX * TY;
// record: [patch headers {blocks, byte offset}] [w0 + potential, as pairs, tile row-major]
// [point index, tile row-major] [blocks: {atom} + projector values [16][4]]
constexpr int REC_V = 128;                 // [point] (w0 + V, w0 + V): the star's centre weight plus the potential
constexpr int REC_IDX = REC_V + NPOS * 8;
constexpr int REC_BLK = REC_IDX + NPOS * 4;
constexpr int BLK = 16 + 16 * 16;
constexpr int MAX_REC = 48 * 1024;         // record slot budget (bytes)
constexpr size_t MAX_SMEM = 226 * 1024;    // dynamic shared memory per CTA (227 KB less the static part)
constexpr int MAX_SLAB = 1 << 16;          // planes per z-slab (at most)
constexpr int MAX_UNITS = 64;              // units per CTA (shared-memory table)
constexpr int SUSPEND_NS = 20000;          // suspension limit of one barrier test
constexpr int SPIN = 100000;               // barrier tests before a wait gives up (default)
constexpr int DRAIN_SPIN = 5000;           // barrier tests per slot when draining after a timeout

// Window layout in a slot.  Window rows wy = 0..15 (tile rows at 4..11),
// columns wx = 0..23 (tile columns at 4..19).  Columns 4..19 of every row
// are positions wy * 16 + wx - 4 (0..255); columns 0..3 and 20..23 of the
// tile rows are positions 256 + (wy - 4) * 8 + (0..3 | 4..7).  Brick row g
// covers positions 4 g .. 4 g + 3: g < 64 row g / 4 of the core columns,
// g >= 64 the side halo.
__host__ __device__ __forceinline__ void group_pos(int g, int &wy, int &wx) {
    if (g < 64) {
        wy = g >> 2;
        wx = 4 + 4 * (g & 3);
    } else {
        const int h = g - 64;
        wy = 4 + (h >> 1);
        wx = (h & 1) ? 20 : 0;
    }
}
// brick rows of the tile itself (window rows 4..11, core columns)
constexpr int G_TILE0 = 16, G_TILE1 = 48;

// A unit as the kernel walks it: planes zm0..zm1 (the slab's output planes
// zo0..zo1-1 and up to four on either side), record / descriptor index of
// plane z = pz + z.
struct UnitDev {
    int zm0, zm1, zo0, zo1, pz, pad0, pad1, pad2;
};

struct Args {
    const UnitDev *units;   // per CTA, concatenated
    const int4 *cta;        // [CTA]: first unit, unit count, first atom, atom count
    const int *cta_atoms;   // per CTA, concatenated: the atoms its records name (in local order)
    const uint32_t *desc;   // [plane][80]: first point | presence mask << 28
    const uint2 *recs;      // [plane]: {offset / 16, bytes}
    const unsigned char *rec;
    const float *psi;       // [npts][ldp]
    int64_t ldp;
    const float *cproj;     // [atom][nb][4]
    float *hpsi;
    int64_t ldh;
    int nb, rec_slot, cs_atoms;   // cs_atoms: the largest atom count of a CTA
    int spin;                     // barrier tests before a wait gives up
    int npts;                     // point count (the bounds-checked build tests indices against it)
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
// at most `spin` tests (by default about SPIN * SUSPEND_NS, two seconds, in all)
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, int spin) {
    for (int i = 0; i < spin; ++i)
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
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Per-thread constants.  Offsets are in float2 units (one state pair) from
// a slot's start.
struct Lane {
    float2 W1, W2, W3, W4;
    int cb;        // centre of patch row 0, column 0 (window row 4 + ty0)
    int lb0, lb1;  // first of the four axis-2 neighbours left of rows 0 / 1
    int rb0, rb1;  // first of the four right of rows 0 / 1
    int to;        // tile index of patch row 0, column 0 (record tables)
    int w, h, sl;
    int npts;      // point count and status word (bounds-checked build)
    int *status;
};

// position p -> float2 offset of the lane's state pair: p * PS + lane
constexpr int PS = ROWB / 8;

// The plane's own terms of its output (everything but the z-terms): the
// centre of the star with the potential, the in-plane star and the
// nonlocal gather, for the patch rows r and columns x of this thread.
__device__ __forceinline__ void plane_terms(float2 (&T)[2][4], const float2 (&cc)[2][4], const float2 *__restrict__ P,
                                            const unsigned char *__restrict__ rs, const float2 *__restrict__ cs,
                                            const Lane &c) {
    const float4 *V4 = reinterpret_cast<const float4 *>(rs + REC_V) + (c.to >> 1);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float4 v01 = V4[r * (TX / 2)], v23 = V4[r * (TX / 2) + 1];
        T[r][0] = make_float2(v01.x, v01.y) * cc[r][0];
        T[r][1] = make_float2(v01.z, v01.w) * cc[r][1];
        T[r][2] = make_float2(v23.x, v23.y) * cc[r][2];
        T[r][3] = make_float2(v23.z, v23.w) * cc[r][3];
    }
    // axis-2 neighbours: the four left and right of each patch row
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float2 v[12];
        const int lb = r ? c.lb1 : c.lb0, rb = r ? c.rb1 : c.rb0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = P[lb + k * PS];
            v[8 + k] = P[rb + k * PS];
            v[4 + k] = cc[r][k];
        }
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            const float2 W = j == 1 ? c.W1 : j == 2 ? c.W2 : j == 3 ? c.W3 : c.W4;
#pragma unroll
            for (int x = 0; x < 4; ++x) T[r][x] = fma2(W, add2(v[x + 4 + j], v[x + 4 - j]), T[r][x]);
        }
    }
    // axis-1 neighbours: window rows ty0 .. ty0 + 9 of each patch column,
    // summed apart from the rest (shorter dependent chains) and added at the end
    float2 Ty[2][4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        float2 y[10];
#pragma unroll
        for (int m = 0; m < 10; ++m) {
            if (m == 4 || m == 5) y[m] = cc[m - 4][x];
            else y[m] = P[c.cb + ((m - 4) * 16 + x) * PS];
        }
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            const float2 W = j == 1 ? c.W1 : j == 2 ? c.W2 : j == 3 ? c.W3 : c.W4;
#pragma unroll
            for (int r = 0; r < 2; ++r)
                Ty[r][x] = j == 1 ? W * add2(y[r + 4 + j], y[r + 4 - j])
                                  : fma2(W, add2(y[r + 4 + j], y[r + 4 - j]), Ty[r][x]);
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int x = 0; x < 4; ++x) T[r][x] = add2(T[r][x], Ty[r][x]);
    // nonlocal gather: per atom meeting the patch, the projection
    // coefficients of the lane's two states (staged in shared memory)
    // against the patch's projector values (scalar FMAs: a projector value
    // multiplies both states without being paired with itself first)
    const int2 hd = reinterpret_cast<const int2 *>(rs)[c.w];
    const unsigned char *blk = rs + hd.y;
    for (int k = 0; k < hd.x; ++k, blk += BLK) {
        const float2 *cq = cs + *reinterpret_cast<const int *>(blk) * (4 * SG / 2) + c.sl;
        const float2 c0 = cq[0], c1 = cq[SG / 2], c2 = cq[SG], c3 = cq[3 * SG / 2];
        const float4 *g = reinterpret_cast<const float4 *>(blk + 16) + 8 * c.h;
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const float4 gv = g[r * 4 + x];
                float2 a = T[r][x];
                a.x = __fmaf_rn(gv.x, c0.x, a.x);
                a.y = __fmaf_rn(gv.x, c0.y, a.y);
                a.x = __fmaf_rn(gv.y, c1.x, a.x);
                a.y = __fmaf_rn(gv.y, c1.y, a.y);
                a.x = __fmaf_rn(gv.z, c2.x, a.x);
                a.y = __fmaf_rn(gv.z, c2.y, a.y);
                a.x = __fmaf_rn(gv.w, c3.x, a.x);
                a.y = __fmaf_rn(gv.w, c3.y, a.y);
                T[r][x] = a;
            }
    }
}

// A point index the kernel may store to or copy from (always true unless
// the bounds-checked build finds it out of range, which it records).
__device__ __forceinline__ bool index_ok(int i, int npts, int *status) {
#if RS_BOUNDS_CHECK
    if (i >= npts) {
        atomicOr(status, 2);
        return false;
    }
#endif
    return true;
}

// Writes the finished output of the plane in accumulator slot R.
template <int R>
__device__ __forceinline__ void emit(const float2 (&A)[8][2][4], const int *rowring, float *hp, int64_t ldh,
                                     const Lane &c) {
    const int4 *ring4 = reinterpret_cast<const int4 *>(rowring + R * NPOS) + (c.to >> 2);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int4 id = ring4[r * (TX / 4)];
#if RS_BOUNDS_CHECK
        if (!index_ok(id.x, c.npts, c.status)) id.x = -1;
        if (!index_ok(id.y, c.npts, c.status)) id.y = -1;
        if (!index_ok(id.z, c.npts, c.status)) id.z = -1;
        if (!index_ok(id.w, c.npts, c.status)) id.w = -1;
#endif
        if (id.x >= 0) *reinterpret_cast<float2 *>(hp + (int64_t)id.x * ldh) = A[R][r][0];
        if (id.y >= 0) *reinterpret_cast<float2 *>(hp + (int64_t)id.y * ldh) = A[R][r][1];
        if (id.z >= 0) *reinterpret_cast<float2 *>(hp + (int64_t)id.z * ldh) = A[R][r][2];
        if (id.w >= 0) *reinterpret_cast<float2 *>(hp + (int64_t)id.w * ldh) = A[R][r][3];
    }
}

// The z-terms of plane z (R = z mod 8): slot k holds output z' = k mod 8 for
// z' = z - 4 .. z + 3 before the step.  Plane z is the last contribution to
// output z - 4, which is then written (when `store`), and its slot takes
// output z + 4, whose first contribution plane z is.
template <int R>
__device__ __forceinline__ void zterms(float2 (&A)[8][2][4], const float2 (&cc)[2][4], const float2 (&T)[2][4],
                                       bool full, bool store, const int *rowring, float *hp, int64_t ldh,
                                       const Lane &c) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const float2 v = cc[r][x];
            A[(R + 4) % 8][r][x] = fma2(c.W4, v, A[(R + 4) % 8][r][x]);
            A[(R + 1) % 8][r][x] = fma2(c.W1, v, A[(R + 1) % 8][r][x]);
            A[(R + 7) % 8][r][x] = fma2(c.W1, v, A[(R + 7) % 8][r][x]);
            A[(R + 2) % 8][r][x] = fma2(c.W2, v, A[(R + 2) % 8][r][x]);
            A[(R + 6) % 8][r][x] = fma2(c.W2, v, A[(R + 6) % 8][r][x]);
            A[(R + 3) % 8][r][x] = fma2(c.W3, v, A[(R + 3) % 8][r][x]);
            A[(R + 5) % 8][r][x] = fma2(c.W3, v, A[(R + 5) % 8][r][x]);
            if (full) A[R][r][x] = add2(A[R][r][x], T[r][x]);
        }
    if (store) emit<(R + 4) % 8>(A, rowring, hp, ldh, c);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int x = 0; x < 4; ++x) A[(R + 4) % 8][r][x] = c.W4 * cc[r][x];
}

__device__ __forceinline__ void emit_any(int r, const float2 (&A)[8][2][4], const int *rowring, float *hp,
                                         int64_t ldh, const Lane &c) {
    switch (r) {
        case 0: emit<0>(A, rowring, hp, ldh, c); break;
        case 1: emit<1>(A, rowring, hp, ldh, c); break;
        case 2: emit<2>(A, rowring, hp, ldh, c); break;
        case 3: emit<3>(A, rowring, hp, ldh, c); break;
        case 4: emit<4>(A, rowring, hp, ldh, c); break;
        case 5: emit<5>(A, rowring, hp, ldh, c); break;
        case 6: emit<6>(A, rowring, hp, ldh, c); break;
        default: emit<7>(A, rowring, hp, ldh, c); break;
    }
}

// Position of the CTA in its unit list: unit k (a copy in U), plane z.
struct Cursor {
    int k, z;
    UnitDev U;
};

template <int RING>
__global__ void __launch_bounds__(NT, 1) k_hpsi_ring(Args a) {
    static_assert(AHEAD < RING, "copy distance must leave a slot to compute on");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint64_t fullb[RING], emptyb[RING];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = blockIdx.y;
    const int4 mine = a.cta[blockIdx.x];   // first unit, units, first atom, atoms
    const int nu = min(mine.y, MAX_UNITS);
    unsigned char *psi_ring = smraw;                                       // [RING] windows
    unsigned char *rec_ring = smraw + (size_t)RING * SLOT_PSI;            // [RING] records
    float *cs = reinterpret_cast<float *>(rec_ring + (size_t)RING * a.rec_slot);   // [atom][4][32]
    UnitDev *ut = reinterpret_cast<UnitDev *>(cs + (size_t)a.cs_atoms * 4 * SG);   // [MAX_UNITS]
    int *rowring = reinterpret_cast<int *>(ut + MAX_UNITS);               // [8][NPOS] output rows
    if (tid == 0) {
        for (int i = 0; i < RING; ++i) {
            bar_init(&fullb[i], NT);    // every thread's copy completions
            bar_init(&emptyb[i], NW);   // every warp's release
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int k = tid; k < nu; k += NT) ut[k] = a.units[mine.x + k];
    // projection coefficients of the CTA's atoms, [local atom][projector][state]
    for (int e = tid; e < mine.w * 4 * SG; e += NT) {
        const int la = e >> 7, q = (e >> 5) & 3, st = e & 31;
        const int at = __ldg(a.cta_atoms + mine.z + la);
        cs[e] = __ldg(a.cproj + ((int64_t)at * a.nb + grp * SG + st) * 4 + q);
    }
    __syncthreads();
    if (nu == 0) return;

    // ---- copies: plane qi into slot j % RING.  Lane l of warp w copies
    // bytes 16 (l % 8) .. of position l / 8 of brick rows w + 8 k.  The
    // descriptors of the next three planes to copy are held by lane groups
    // 0..9, 10..19, 20..29 (plane j in group j mod 3, brick row w + 8 (lane
    // mod 10)), their record addresses by lanes 0, 10, 20; a group is
    // reloaded, for plane j + 3 (cursor qd), as soon as plane j is issued.
    bool ok = true;
    const float *src0 = a.psi + grp * SG + 4 * (lane & 7);
    const int doff = (4 * warp + (lane >> 3)) * ROWB + 16 * (lane & 7);   // + k * 32 * ROWB
    const uint32_t rbit = 1u << (lane >> 3);
    const int lgrp = lane < 30 ? lane / 10 : -1, lsub = lane % 10;
    uint32_t dq = 0u;
    uint2 rq = make_uint2(0u, 0u);
    auto advance = [&](Cursor &q) {
        if (++q.z > q.U.zm1) {
            ++q.k;
            if (q.k < nu) {
                q.U = ut[q.k];
                q.z = q.U.zm0;
            }
        }
    };
    auto load_desc = [&](const Cursor &q, int g) {
        if (q.k < nu && lgrp == g) {
            const int64_t pt = (int64_t)q.U.pz + q.z;
            dq = __ldg(a.desc + pt * NG + warp + NW * lsub);
            if (lsub == 0) rq = (q.z >= q.U.zo0 && q.z < q.U.zo1) ? __ldg(a.recs + pt) : make_uint2(0u, 0u);
        }
    };
    Cursor qi{0, ut[0].zm0, ut[0]}, qc = qi, qd = qi;
    for (int g = 0; g < 3; ++g) {
        load_desc(qd, g);
        if (qd.k < nu) advance(qd);
    }
    int j = 0;   // planes issued
    auto issue = [&]() {
        const int slot = j % RING, g = j % 3;
        if (!__all_sync(0xffffffffu, j < RING || bar_wait(&emptyb[slot], ((j / RING) - 1) & 1, a.spin))) {
            ok = false;
            return;
        }
        const bool pfull = qi.z >= qi.U.zo0 && qi.z < qi.U.zo1;
        unsigned char *dst = psi_ring + (size_t)slot * SLOT_PSI + doff;
#pragma unroll
        for (int k = 0; k < CPW; ++k) {
            // edge planes: the tile's own brick rows only (16 .. 47)
            if (!pfull && (k < G_TILE0 / NW || k >= G_TILE1 / NW)) continue;
            const uint32_t d = __shfl_sync(0xffffffffu, dq, 10 * g + k);
            const uint32_t mask = d >> 28;
            const bool has = (mask & rbit) != 0;
            const int pnt = (int)(d & 0x0fffffffu) + __popc(mask & (rbit - 1u));
            const bool use = has && index_ok(pnt, a.npts, a.status);
            cp_async16(dst + k * (NW * 4 * ROWB), use ? src0 + (int64_t)pnt * a.ldp : src0, use);
        }
        if (pfull) {
            const uint32_t rx = __shfl_sync(0xffffffffu, rq.x, 10 * g), ry = __shfl_sync(0xffffffffu, rq.y, 10 * g);
            const unsigned char *rsrc = a.rec + (size_t)rx * 16;
            unsigned char *rdst = rec_ring + (size_t)slot * a.rec_slot;
            for (int o = tid * 16; o < (int)ry; o += NT * 16) cp_async16(rdst + o, rsrc + o, true);
        }
        cp_async_arrive(&fullb[slot]);
        ++j;
        advance(qi);
        load_desc(qd, g);
        if (qd.k < nu) advance(qd);
    };

    Lane c;
    c.W1 = f2(a.w[1]);
    c.W2 = f2(a.w[2]);
    c.W3 = f2(a.w[3]);
    c.W4 = f2(a.w[4]);
    c.w = warp;
    c.h = lane >> 4;
    c.sl = lane & 15;
    c.npts = a.npts;
    c.status = a.status;
    {
        const int px = warp & 3, ty0 = 4 * (warp >> 2) + 2 * c.h, sl = c.sl;
        const int tx0 = 4 * px;
        c.cb = ((ty0 + 4) * 16 + tx0) * PS + sl;
        c.to = ty0 * TX + tx0;
        // left / right neighbours: core columns, or the side halo at the tile's edges
        c.lb0 = (px == 0 ? 256 + ty0 * 8 : (ty0 + 4) * 16 + tx0 - 4) * PS + sl;
        c.lb1 = (px == 0 ? 256 + (ty0 + 1) * 8 : (ty0 + 5) * 16 + tx0 - 4) * PS + sl;
        c.rb0 = (px == 3 ? 256 + ty0 * 8 + 4 : (ty0 + 4) * 16 + tx0 + 4) * PS + sl;
        c.rb1 = (px == 3 ? 256 + (ty0 + 1) * 8 + 4 : (ty0 + 5) * 16 + tx0 + 4) * PS + sl;
    }
    const float2 *cs2 = reinterpret_cast<const float2 *>(cs);
    float *hp = a.hpsi + grp * SG + 2 * c.sl;
    float2 A[8][2][4];

    while (j < AHEAD && qi.k < nu && ok) issue();
    int it = 0;   // planes consumed
    for (; qc.k < nu && ok; ++it) {
        if (qi.k < nu) {
            issue();
            if (!ok) break;
        }
        const int slot = it % RING;
        if (!__all_sync(0xffffffffu, bar_wait(&fullb[slot], (it / RING) & 1, a.spin))) {
            ok = false;
            break;
        }
        const UnitDev &U = qc.U;
        const int z = qc.z;
        if (z == U.zm0) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int x = 0; x < 4; ++x) A[k][r][x] = make_float2(0.f, 0.f);
        }
        const bool full = z >= U.zo0 && z < U.zo1;
        const float2 *P = reinterpret_cast<const float2 *>(psi_ring + (size_t)slot * SLOT_PSI);
        const unsigned char *rs = rec_ring + (size_t)slot * a.rec_slot;
        float2 cc[2][4], T[2][4];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int x = 0; x < 4; ++x) cc[r][x] = P[c.cb + (r * 16 + x) * PS];
        if (full) {
            plane_terms(T, cc, P, rs, cs2, c);
            // the plane's point indices to the output ring (one lane per half-warp)
            if (c.sl == 0) {
                const int4 *I4 = reinterpret_cast<const int4 *>(rs + REC_IDX) + (c.to >> 2);
                int4 *ring4 = reinterpret_cast<int4 *>(rowring + (z & 7) * NPOS) + (c.to >> 2);
                ring4[0] = I4[0];
                ring4[TX / 4] = I4[TX / 4];
            }
        }
        __syncwarp();
        if (lane == 0) bar_arrive(&emptyb[slot]);   // the slot is no longer read by this warp
        const bool st = z - 4 >= U.zo0 && z - 4 < U.zo1;
        switch (z & 7) {
            case 0: zterms<0>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
            case 1: zterms<1>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
            case 2: zterms<2>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
            case 3: zterms<3>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
            case 4: zterms<4>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
            case 5: zterms<5>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
            case 6: zterms<6>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
            default: zterms<7>(A, cc, T, full, st, rowring, hp, a.ldh, c); break;
        }
        // last plane of the column inside the unit: planes beyond it are
        // empty, so the outputs still open are complete
        if (z == U.zm1 && z < U.zo1 + 3) {
            for (int o = z - 3; o <= z; ++o)
                if (o >= U.zo0 && o < U.zo1) emit_any(o & 7, A, rowring, hp, a.ldh, c);
        }
        advance(qc);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (!ok) {
        if (lane == 0) atomicExch(a.status, 1);
        // A wait gave up.  The planes this thread issued but did not consume
        // (at most RING, in distinct slots) may still have arrivals pending
        // from its copies; wait for their phases, with a fixed bound, so that
        // no asynchronous arrival reaches shared memory after the CTA exits.
        for (int q = it; q < j; ++q) bar_wait(&fullb[q % RING], (q / RING) & 1, DRAIN_SPIN);
    }
}

}  // namespace

struct RingPlan {
    DevBuf units, cta, cta_atoms, desc, recs, rec, status;
    int n_cta = 0, rec_slot = 0, cs_atoms = 0, ring = MAX_RING, spin = SPIN;
    int64_t nplanes = 0;
    float w0 = 0.f;
    int64_t npts = 0;
    size_t smem = 0;
};

void ring_plan_destroy(RingPlan *p) { delete p; }

int ring_plan_build(RingPlan **out, const rs_grid *g, const std::vector<int32_t> &coff, const std::vector<int32_t> &catom,
                    const std::vector<float> &cg32, const std::vector<float> &v32, float w0, int n_atoms, int slab) {
    (void)n_atoms;
    *out = nullptr;
    // the descriptors describe four consecutive points per brick row: the
    // kernel needs the order of bricks of 4^3 points
    if (g->order != 4 || g->npts >= (1 << 28) || slab < 1 || slab > MAX_SLAB) return RS_OK;
    const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
    auto at = [&](int a0, int a1, int a2) -> int32_t {
        if (a0 < 0 || a1 < 0 || a2 < 0 || a0 >= d0 || a1 >= d1 || a2 >= d2) return -1;
        return g->map[((size_t)a0 * d1 + a1) * d2 + a2];
    };
    const int n1 = (d1 + TY - 1) / TY, n2 = (d2 + TX - 1) / TX;
    struct Col {
        int zmin, zmax;
        int64_t p0;   // record / descriptor index of plane zmin
    };
    std::vector<Col> cols;
    std::vector<uint32_t> desc;
    std::vector<uint2> recs;
    std::vector<double> pcost;   // march cost of each full plane (planes of the nonlocal-heaviest patch cost more)
    std::vector<int32_t> blob;   // 4-byte words; records start on 16-byte boundaries
    int max_rec = 0;
    int64_t nplanes = 0;
    auto word = [](float f) {
        int32_t b;
        memcpy(&b, &f, 4);
        return b;
    };
    try {
        for (int t1 = 0; t1 < n1; ++t1)
            for (int t2 = 0; t2 < n2; ++t2) {
                const int b1 = t1 * TY, b2 = t2 * TX;
                int zmin = d0, zmax = -1;
                for (int a0 = 0; a0 < d0; ++a0)
                    for (int iy = 0; iy < TY; ++iy)
                        for (int ix = 0; ix < TX; ++ix)
                            if (at(a0, b1 + iy, b2 + ix) >= 0) {
                                zmin = std::min(zmin, a0);
                                zmax = std::max(zmax, a0);
                            }
                if (zmax < 0) continue;
                cols.push_back({zmin, zmax, nplanes});
                for (int z = zmin; z <= zmax; ++z) {
                    for (int gi = 0; gi < NG; ++gi) {
                        int wy, wx;
                        group_pos(gi, wy, wx);
                        uint32_t mask = 0;
                        int32_t first = -1, prev = -1;
                        for (int i = 0; i < 4; ++i) {
                            const int32_t m = at(z, b1 + wy - 4, b2 + wx - 4 + i);
                            if (m < 0) continue;
                            if (first < 0) first = m;
                            else if (m != prev + 1) return fail(RS_EINVAL, "stencil plan: brick row not consecutive");
                            prev = m;
                            mask |= 1u << i;
                        }
                        desc.push_back((mask << 28) | (uint32_t)(first < 0 ? 0 : first));
                    }
                    // record of plane z
                    const size_t off = blob.size();
                    std::vector<int32_t> hdr(REC_V / 4, 0), vv(2 * NPOS, 0), ii(NPOS, -1), blocks;
                    for (int iy = 0; iy < TY; ++iy)
                        for (int ix = 0; ix < TX; ++ix) {
                            const int32_t m = at(z, b1 + iy, b2 + ix);
                            if (m < 0) continue;
                            // the centre weight plus the potential, as the kernel would add them
                            const float vw = w0 + v32[m];
                            vv[2 * (iy * TX + ix)] = vv[2 * (iy * TX + ix) + 1] = word(vw);
                            ii[iy * TX + ix] = m;
                        }
                    for (int w = 0; w < NW; ++w) {
                        const int py = w >> 2, px = w & 3;
                        // atom -> projector values of the 16 patch points
                        std::map<int32_t, std::vector<float>> per_atom;
                        for (int rr = 0; rr < 4; ++rr)
                            for (int xx = 0; xx < 4; ++xx) {
                                const int32_t m = ii[(4 * py + rr) * TX + 4 * px + xx];
                                if (m < 0) continue;
                                for (int e = coff[m]; e < coff[m + 1]; ++e) {
                                    std::vector<float> &gv = per_atom[catom[e]];
                                    if (gv.empty()) gv.assign(64, 0.f);
                                    for (int q = 0; q < 4; ++q) gv[(rr * 4 + xx) * 4 + q] = cg32[(size_t)e * 4 + q];
                                }
                            }
                        hdr[2 * w] = (int32_t)per_atom.size();
                        hdr[2 * w + 1] = REC_BLK + (int32_t)blocks.size() * 4;
                        for (const auto &pa : per_atom) {
                            blocks.push_back(pa.first);
                            blocks.push_back(0);
                            blocks.push_back(0);
                            blocks.push_back(0);
                            for (float f : pa.second) blocks.push_back(word(f));
                        }
                    }
                    blob.insert(blob.end(), hdr.begin(), hdr.end());
                    blob.insert(blob.end(), vv.begin(), vv.end());
                    blob.insert(blob.end(), ii.begin(), ii.end());
                    blob.insert(blob.end(), blocks.begin(), blocks.end());
                    const int bytes = (int)((blob.size() - off) * 4);
                    max_rec = std::max(max_rec, bytes);
                    if (off / 4 > UINT32_MAX) return RS_OK;
                    recs.push_back(make_uint2((uint32_t)(off / 4), (uint32_t)bytes));
                    int maxblk = 0;
                    for (int w = 0; w < NW; ++w) maxblk = std::max(maxblk, hdr[2 * w]);
                    pcost.push_back(1.0 + NL_COST * maxblk);
                    ++nplanes;
                }
            }
        if (cols.empty() || max_rec > MAX_REC) return RS_OK;
        int dev = 0, n_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return fail(RS_ECUDA, "device query failed");
        // Units slab by slab, columns in raster order within a slab; the
        // sequence is cut into one contiguous run per CTA of equal modelled
        // cost (an output plane costs 1 plus NL_COST per nonlocal block of its
        // heaviest patch, an edge plane EDGE_COST), a unit split at a plane
        // where a run ends.
        const int G = std::max(1, n_sm);
        struct Piece {
            int zmin, zmax, zo0, zo1;
            int64_t pz;
        };
        std::vector<Piece> seq;
        const int nslab = (d0 + slab - 1) / slab;
        for (int sl = 0; sl < nslab; ++sl)
            for (const Col &cl : cols) {
                const int zo0 = std::max(cl.zmin, sl * slab), zo1 = std::min(cl.zmax + 1, (sl + 1) * slab);
                if (zo0 < zo1) seq.push_back({cl.zmin, cl.zmax, zo0, zo1, cl.p0 - cl.zmin});
            }
        auto edges = [](const Piece &u, int a, int b) {   // edge planes of output planes [a, b)
            return EDGE_COST * ((a - std::max(u.zmin, a - 4)) + (std::min(u.zmax, b + 3) - b + 1));
        };
        double total = 0;
        for (const Piece &u : seq) {
            total += edges(u, u.zo0, u.zo1);
            for (int z = u.zo0; z < u.zo1; ++z) total += pcost[(size_t)(u.pz + z)];
        }
        // Greedy fill of runs up to a cost T (a run takes whole planes while
        // it stays within T; a plane that fits no run alone opens one); the
        // smallest T that needs at most G runs, by bisection.
        std::vector<std::vector<UnitDev>> per;
        auto fill = [&](double T, bool keep) -> int {
            if (keep) per.assign(1, {});
            int runs = 1;
            double load = 0;
            for (const Piece &u : seq) {
                int a = u.zo0;
                while (a < u.zo1) {
                    double c = edges(u, a, a + 1) + pcost[(size_t)(u.pz + a)];
                    if (load > 0 && load + c > T) {
                        ++runs;
                        if (keep) per.emplace_back();
                        load = 0;
                        continue;
                    }
                    int b = a + 1;
                    while (b < u.zo1) {
                        const double nc = c - edges(u, a, b) + edges(u, a, b + 1) + pcost[(size_t)(u.pz + b)];
                        if (load + nc > T) break;
                        c = nc;
                        ++b;
                    }
                    if (keep) {
                        UnitDev d{};
                        d.zo0 = a;
                        d.zo1 = b;
                        d.zm0 = std::max(u.zmin, a - 4);
                        d.zm1 = std::min(u.zmax, b + 3);
                        d.pz = (int)u.pz;
                        per.back().push_back(d);
                    }
                    load += c;
                    a = b;
                    if (a < u.zo1) {
                        ++runs;
                        if (keep) per.emplace_back();
                        load = 0;
                    }
                }
            }
            return runs;
        };
        for (const Piece &u : seq)
            if (u.pz < INT32_MIN || u.pz > INT32_MAX) return RS_OK;
        double lo = total / G, hi = 2.0 * total / G + 16.0;
        for (int i = 0; i < 50; ++i) {
            const double mid = 0.5 * (lo + hi);
            if (fill(mid, false) <= G) hi = mid;
            else lo = mid;
        }
        fill(hi, true);
        if ((int)per.size() > G) return RS_OK;
        per.resize(G);
        // per CTA: the atoms its records name, renumbered in the records to
        // the CTA's local order (a record belongs to the one unit whose
        // output planes hold it)
        std::vector<UnitDev> flat;
        std::vector<int4> cta(G);
        std::vector<int32_t> cta_atoms;
        int cs_atoms = 0;
        for (int k = 0; k < G; ++k) {
            if (per[k].size() > (size_t)MAX_UNITS) return RS_OK;
            std::map<int32_t, int32_t> local;
            const int first_atom = (int)cta_atoms.size();
            for (const UnitDev &u : per[k])
                for (int z = u.zo0; z < u.zo1; ++z) {
                    const size_t w0 = (size_t)recs[(size_t)((int64_t)u.pz + z)].x * 4;
                    for (int w = 0; w < NW; ++w) {
                        const int cnt = blob[w0 + 2 * w], b0 = blob[w0 + 2 * w + 1];
                        for (int q = 0; q < cnt; ++q) {
                            int32_t &aw = blob[w0 + (size_t)(b0 + q * BLK) / 4];
                            auto it = local.find(aw);
                            if (it == local.end()) {
                                it = local.emplace(aw, (int32_t)local.size()).first;
                                cta_atoms.push_back(aw);
                            }
                            aw = it->second;
                        }
                    }
                }
            cs_atoms = std::max(cs_atoms, (int)local.size());
            cta[k] = make_int4((int)flat.size(), (int)per[k].size(), first_atom, (int)local.size());
            flat.insert(flat.end(), per[k].begin(), per[k].end());
        }
        if (cta_atoms.empty()) cta_atoms.push_back(0);
        RingPlan *P = new (std::nothrow) RingPlan;
        if (!P) return fail(RS_ENOMEM, "host allocation failed");
        auto bail = [&](int rc) {
            delete P;
            return rc;
        };
        int rc;
        if ((rc = P->units.upload(flat.data(), flat.size() * sizeof(UnitDev))) ||
            (rc = P->cta.upload(cta.data(), cta.size() * sizeof(int4))) ||
            (rc = P->cta_atoms.upload(cta_atoms.data(), cta_atoms.size() * sizeof(int32_t))) ||
            (rc = P->desc.upload(desc.data(), desc.size() * sizeof(uint32_t))) ||
            (rc = P->recs.upload(recs.data(), recs.size() * sizeof(uint2))) ||
            (rc = P->rec.upload(blob.data(), blob.size() * sizeof(int32_t))) || (rc = P->status.alloc(sizeof(int))))
            return bail(rc);
        if (cudaMemset(P->status.p, 0, sizeof(int)) != cudaSuccess) return bail(fail(RS_ECUDA, "cudaMemset failed"));
        P->n_cta = G;
        P->nplanes = nplanes;
        P->w0 = w0;
        P->rec_slot = (max_rec + 127) & ~127;
        P->cs_atoms = cs_atoms;
        P->npts = g->npts;
        const size_t fixed = (size_t)cs_atoms * 4 * SG * sizeof(float) + MAX_UNITS * sizeof(UnitDev) + 8 * NPOS * sizeof(int);
        for (P->ring = MAX_RING; P->ring > AHEAD; --P->ring) {
            P->smem = (size_t)P->ring * (SLOT_PSI + P->rec_slot) + fixed;
            if (P->smem <= MAX_SMEM) break;
        }
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
    a.cta = p->cta.as<int4>();
    a.cta_atoms = p->cta_atoms.as<int>();
    a.cs_atoms = p->cs_atoms;
    a.desc = p->desc.as<uint32_t>();
    a.recs = p->recs.as<uint2>();
    a.rec = p->rec.as<unsigned char>();
    a.psi = psi;
    a.ldp = ldp;
    a.cproj = cproj;
    a.hpsi = hpsi;
    a.ldh = ldh;
    a.nb = nb;
    a.rec_slot = p->rec_slot;
    a.spin = p->spin;
    a.npts = (int)p->npts;
    for (int j = 0; j < 5; ++j) a.w[j] = w[j];
    a.status = p->status.as<int>();
    const dim3 grid((unsigned)p->n_cta, (unsigned)(nb / SG));
    const int r4 = p->ring == 4 ? 1 : 0;
    RS_TRY(smem_optin(r4 ? (const void *)k_hpsi_ring<4> : (const void *)k_hpsi_ring<3>, p->smem));
    if (r4) k_hpsi_ring<4><<<grid, NT, p->smem, st>>>(a);
    else k_hpsi_ring<3><<<grid, NT, p->smem, st>>>(a);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

int ring_status(const RingPlan *p, int *flag) {
    *flag = 0;
    if (!p) return RS_OK;
    RS_CUDA(cudaMemcpy(flag, p->status.as<int>(), sizeof(int), cudaMemcpyDeviceToHost));
    return RS_OK;
}

// the (w0 + V, w0 + V) pairs of every plane record from a new FP32
// potential (the same FP32 sum the plan builder forms on the host)
__global__ void k_ring_potential(const uint2 *__restrict__ recs, int64_t nplanes, unsigned char *__restrict__ rec,
                                 const float *__restrict__ v32, float w0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nplanes * NPOS) return;
    const int64_t plane = t / NPOS;
    const int pos = (int)(t - plane * NPOS);
    unsigned char *r = rec + (size_t)recs[plane].x * 16;
    const int idx = reinterpret_cast<const int *>(r + REC_IDX)[pos];
    if (idx < 0) return;
    const float vw = __fadd_rn(w0, v32[idx]);
    reinterpret_cast<float2 *>(r + REC_V)[pos] = make_float2(vw, vw);
}

int ring_set_potential(RingPlan *p, const float *v32, cudaStream_t st) {
    if (!p) return RS_OK;
    const int64_t n = p->nplanes * NPOS;
    k_ring_potential<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p->recs.as<uint2>(), p->nplanes,
                                                                  p->rec.as<unsigned char>(), v32, p->w0);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

int ring_reset_status(RingPlan *p) {
    if (!p) return RS_OK;
    RS_CUDA(cudaMemset(p->status.p, 0, sizeof(int)));
    return RS_OK;
}

int *ring_status_word(RingPlan *p) { return p ? p->status.as<int>() : nullptr; }

void ring_set_wait_limit(RingPlan *p, int tests) {
    if (p) p->spin = tests < 0 ? SPIN : tests;
}

}  // namespace rs

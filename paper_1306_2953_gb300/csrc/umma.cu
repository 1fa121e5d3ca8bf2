// Dense contractions of the FP32 mode on the 5th-generation tensor cores.
//
// Both contractions of Sec. VI are written as D[m][n] = sum_k A[m][k] B[n][k]
// ("TN", both operands K-major):
//   overlap   S = dV X^T Y : A = X^T, B = Y^T, K = grid points;
//   rotation  Y = X C      : A = X, B = C^T, K = states.
// FP32 operands are split exactly into three BF16 pieces, x = x0 + x1 + x2
// (8 + 8 + 8 significant bits), by a pre-pass that also lays them out
// K-major; the product sums the six piece products whose weight is at least
// 2^-16 relative (x0y0, x0y1, x1y0, x0y2, x1y1, x2y0) on tcgen05 (kind::f16,
// BF16 inputs, FP32 accumulation in tensor memory).  Every piece product is
// exact in FP32, so the result carries FP32-level rounding of the
// accumulation only.
//
// Kernel: one CTA of 128 threads per 128 x BN output tile and K range.
// A multi-stage pipeline (three stages for BN = 64, two for BN = 128):
// thread 0 streams, by TMA (cp.async.bulk.tensor, 128-byte swizzle), the
// three pieces of a 128 x 64 A tile and a BN x 64 B tile into the next free
// stage; thread 32 waits for a full stage, issues 6 x 4 tcgen05.mma
// (M = 128, K = 16 each) into a TMEM accumulator and commits to the stage's
// "empty" barrier, which frees it for thread 0.  After
// the K range the four warps read the accumulator with tcgen05.ld (warp w owns
// TMEM lanes 32w..32w+31) and apply the epilogue.  Every wait is bounded; on
// a timeout the kernel raises an error flag, skips the rest and still frees
// its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "device.h"
#include "umma.h"

namespace rs {

constexpr int UM_BM = 128, UM_BK = 64, UM_NT = 128;
constexpr int UM_KB_CTA = 32;   // K blocks per CTA of a split-K contraction (2048 points)
// pipeline stages: three of 72 KB for 64-wide tiles, two of 96 KB for 128-wide
__host__ __device__ constexpr int um_stages(int BN) { return BN <= 64 ? 3 : 2; }
constexpr long long UM_SPIN = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < UM_SPIN; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (SBO), LBO unused (1),
// descriptor version 1, layout type 2 (128B swizzle).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                      // leading byte offset (16 B units), unused here
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

struct UmmaArgs {
    int M, N, K;          // logical sizes (D is M x N)
    int kb_per_cta;       // K blocks of 64 per CTA (split K)
    int mode;             // 0: atomically add alpha*D to FP64 S; 1: Y = alpha*D + beta*Y (FP32)
    double alpha, beta;
    double *S;
    int64_t lds;
    float *Y;
    int64_t ldy;
    int yvec;             // mode 1: Y rows 16-byte aligned (Y and ldy multiples of 4 floats)
    int *err;
};

// Split pieces of a piece pair list: (a piece, b piece)
__constant__ int c_pairs[6][2] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};

template <int BN>
__global__ void __launch_bounds__(UM_NT, 1) k_umma_tn(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, UmmaArgs args) {
    constexpr int A_BYTES = 3 * UM_BM * UM_BK * 2, B_BYTES = 3 * BN * UM_BK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    constexpr int NS = um_stages(BN);
    extern __shared__ __align__(1024) unsigned char smraw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[NS], empty[NS], done;
    __shared__ uint32_t tmem_base;
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * UM_BM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * args.kb_per_cta;
    const int nkb_total = (args.K + UM_BK - 1) / UM_BK;
    const int nk = max(0, min(args.kb_per_cta, nkb_total - kb0));
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&done, 1);
        bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(BN < 32 ? 32 : BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    // thread 0 streams the operand tiles NS stages ahead; thread 32 issues
    // the MMAs and releases every stage when its MMAs have read it
    if (tid == 0 && nk > 0) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % NS;
            if (kb >= NS && !mbar_wait(&empty[s], ((kb / NS) - 1) & 1)) {
                bad = 1;
                break;
            }
            unsigned char *sA = base + s * STAGE, *sB = sA + A_BYTES;
            mbar_expect_tx(&full[s], STAGE);
            tma_load_3d(sA, &tmA, &full[s], (kb0 + kb) * UM_BK, m0, 0);
            tma_load_3d(sB, &tmB, &full[s], (kb0 + kb) * UM_BK, n0, 0);
        }
    } else if (tid == 32 && nk > 0) {
        constexpr uint32_t idesc = umma_idesc(UM_BM, BN);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % NS;
            if (!mbar_wait(&full[s], (kb / NS) & 1)) {
                bad = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sA = smem_u32(base + s * STAGE), sB = sA + A_BYTES;
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
                const uint32_t pa = sA + c_pairs[pr][0] * (UM_BM * UM_BK * 2);
                const uint32_t pb = sB + c_pairs[pr][1] * (BN * UM_BK * 2);
#pragma unroll
                for (int k = 0; k < UM_BK / 16; ++k)
                    umma_f16(tmem, umma_desc_sw128(pa + k * 32), umma_desc_sw128(pb + k * 32), idesc,
                             (kb > 0 || pr > 0 || k > 0) ? 1u : 0u);
            }
            umma_commit(&empty[s]);
        }
        umma_commit(&done);
    }
    __syncthreads();
    // epilogue: every warp reads its 32 TMEM lanes (rows m0 + 32 warp + lane)
    bool ok = nk > 0 && !bad && mbar_wait(&done, 0);
    if (!ok && nk > 0 && tid == 0) atomicExch(args.err, 1);
    __syncthreads();
    ok = ok && !bad;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const int m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (m < args.M) {
                if (args.mode == 0) {
                    double *srow = args.S + (int64_t)m * args.lds;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = n0 + c0 + j;
                        if (n < args.N) atomicAdd(srow + n, args.alpha * (double)__uint_as_float(r[j]));
                    }
                } else if (args.yvec && n0 + c0 + 32 <= args.N) {
                    // the thread's 32 columns are 128 contiguous bytes of its row
                    float4 *y4 = reinterpret_cast<float4 *>(args.Y + (int64_t)m * args.ldy + n0 + c0);
                    const float al = (float)args.alpha, be = (float)args.beta;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float4 v = make_float4(al * __uint_as_float(r[4 * j]), al * __uint_as_float(r[4 * j + 1]),
                                               al * __uint_as_float(r[4 * j + 2]), al * __uint_as_float(r[4 * j + 3]));
                        if (args.beta != 0.0) {
                            const float4 o = y4[j];
                            v.x = v.x + be * o.x;
                            v.y = v.y + be * o.y;
                            v.z = v.z + be * o.z;
                            v.w = v.w + be * o.w;
                        }
                        y4[j] = v;
                    }
                } else {
                    float *yrow = args.Y + (int64_t)m * args.ldy;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = n0 + c0 + j;
                        if (n < args.N) {
                            const float v = (float)args.alpha * __uint_as_float(r[j]);
                            yrow[n] = args.beta == 0.0 ? v : v + (float)args.beta * yrow[n];
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(BN < 32 ? 32 : BN)
                     : "memory");
}

__global__ void k_zero_s(double *S, int64_t lds, int n, int m) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * m;
         e += (int64_t)gridDim.x * blockDim.x)
        S[(e / m) * lds + e % m] = 0.0;
}

// ---------------------------------------------------------------- split ---

__device__ __forceinline__ void split3(float x, __nv_bfloat16 &a, __nv_bfloat16 &b, __nv_bfloat16 &c) {
    a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);     // exact
    b = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b);    // exact
    c = __float2bfloat16_rn(r2);
}

// Transposed split: P[piece][c][k] = piece of X[k][c0 + c], k < K (rows), c < C
// (columns); P has row pitch Kp and piece stride C * Kp.  32 x 32 tiles.
template <typename T>
__global__ void k_split_t(const T *__restrict__ X, int64_t ldx, int K, int C, int Kp, __nv_bfloat16 *__restrict__ P) {
    __shared__ float t[32][33];
    const int k0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int k = k0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (k < K && c < C) ? (float)X[(int64_t)k * ldx + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, k = k0 + threadIdx.x;
        if (c < C && k < Kp) {
            __nv_bfloat16 a, b, d;
            split3(k < K ? t[threadIdx.x][i] : 0.f, a, b, d);
            const int64_t o = (int64_t)c * Kp + k;
            P[o] = a;
            P[(int64_t)C * Kp + o] = b;
            P[2 * (int64_t)C * Kp + o] = d;
        }
    }
}

// Direct split: P[piece][r][k] = piece of X[r][k], k < K (padded to Kp, a
// multiple of 64).  Block (64, 4): threadIdx.y picks one of four rows,
// threadIdx.x strides the row's columns.
template <typename T>
__global__ void k_split_n(const T *__restrict__ X, int64_t ldx, int R, int K, int Kp, __nv_bfloat16 *__restrict__ P) {
    const int64_t n = (int64_t)R * Kp;
    for (int r = blockIdx.x * 4 + threadIdx.y; r < R; r += gridDim.x * 4) {
        const T *xr = X + (int64_t)r * ldx;
        __nv_bfloat16 *pr = P + (int64_t)r * Kp;
        for (int k = threadIdx.x; k < Kp; k += 64) {
            __nv_bfloat16 a, b, d;
            split3(k < K ? (float)xr[k] : 0.f, a, b, d);
            pr[k] = a;
            pr[n + k] = b;
            pr[2 * n + k] = d;
        }
    }
}

// ------------------------------------------------------------------ host ---

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;

int encoder(PFN_cuTensorMapEncodeTiled_v12000 *out) {
    std::call_once(g_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    if (!g_encode) return fail(RS_ECUDA, "cuTensorMapEncodeTiled unavailable");
    *out = g_encode;
    return RS_OK;
}

// 3-D map over pieces [3][rows][Kp] (bf16), box {64, box_rows, 3}, 128-byte swizzle
int make_map(CUtensorMap *m, const void *P, int rows, int Kp, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    RS_TRY(encoder(&enc));
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, 3};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
    cuuint32_t box[3] = {UM_BK, (cuuint32_t)box_rows, 3};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(P), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(RS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RS_OK;
}

template <int BN> int launch(const CUtensorMap &ta, const CUtensorMap &tb, const UmmaArgs &a, int splits, cudaStream_t st) {
    constexpr int STAGE = 3 * UM_BM * UM_BK * 2 + 3 * BN * UM_BK * 2;
    const size_t smem = (size_t)um_stages(BN) * STAGE + 1024;
    RS_TRY(smem_optin((const void *)k_umma_tn<BN>, smem));
    dim3 grid((unsigned)((a.M + UM_BM - 1) / UM_BM), (unsigned)((a.N + BN - 1) / BN), (unsigned)splits);
    k_umma_tn<BN><<<grid, UM_NT, smem, st>>>(ta, tb, a);
    RS_LAUNCH_CHECK();
    return RS_OK;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

int64_t umma_work_bytes(int64_t rows_a, int64_t rows_b, int64_t K) {
    const int64_t Kp = round_up(std::max<int64_t>(K, 1), UM_BK);
    return 3 * (round_up(rows_a, UM_BM) + round_up(rows_b, 128)) * Kp * 2 + 4096;
}

// S (nx x ny, FP64, lds) = dV X^T Y for FP32 X [npts][ldx], Y [npts][ldy].
int64_t umma_split_cache_bytes(bool gram, int64_t npts, int64_t ncols) {
    return gram ? 3 * round_up(ncols, UM_BM) * round_up(npts, UM_BK) * 2 : 3 * round_up(npts, UM_BM) * round_up(ncols, UM_BK) * 2;
}

namespace {
bool cache_hit(const UmmaSplitCache *c, const float *X, int n, int64_t ld, int64_t rows) {
    return c && c->buf && c->valid && c->src == X && c->n == n && c->ld == ld && c->rows == rows;
}
void cache_set(UmmaSplitCache *c, const float *X, int n, int64_t ld, int64_t rows) {
    if (!c || !c->buf) return;
    c->src = X;
    c->n = n;
    c->ld = ld;
    c->rows = rows;
    c->valid = true;
}
}  // namespace

int umma_gram(const float *X, int64_t ldx, int nx, const float *Y, int64_t ldy, int ny, int64_t npts, double dV,
              double *S, int64_t lds, void *work, int *err, cudaStream_t st, UmmaSplitCache *xcache) {
    const int64_t Kp = round_up(npts, UM_BK);
    if (Kp > INT32_MAX / 2) return fail(RS_EINVAL, "umma_gram: too many points");
    const int BN = ny <= 64 ? 64 : 128;
    const bool cached = xcache && xcache->buf;
    __nv_bfloat16 *PA = reinterpret_cast<__nv_bfloat16 *>(cached ? xcache->buf : work);
    __nv_bfloat16 *PB = cached ? reinterpret_cast<__nv_bfloat16 *>(work) : PA + 3 * round_up(nx, UM_BM) * Kp;
    dim3 tb(32, 8);
    // S = X^T X: one split serves both operands
    const bool same = X == Y && ldx == ldy && nx == ny;
    if (same) PB = PA;
    if (!cache_hit(xcache, X, nx, ldx, npts)) {
        k_split_t<float><<<dim3((unsigned)(Kp / 32), (unsigned)((nx + 31) / 32)), tb, 0, st>>>(X, ldx, (int)npts, nx,
                                                                                             (int)Kp, PA);
        cache_set(xcache, X, nx, ldx, npts);
    }
    if (!same)
        k_split_t<float><<<dim3((unsigned)(Kp / 32), (unsigned)((ny + 31) / 32)), tb, 0, st>>>(Y, ldy, (int)npts, ny, (int)Kp,
                                                                                             PB);
    RS_LAUNCH_CHECK();
    CUtensorMap ta, tbm;
    RS_TRY(make_map(&ta, PA, nx, (int)Kp, UM_BM));
    RS_TRY(make_map(&tbm, PB, ny, (int)Kp, BN));
    k_zero_s<<<64, 256, 0, st>>>(S, lds, nx, ny);
    UmmaArgs a{};
    a.M = nx;
    a.N = ny;
    a.K = (int)Kp;
    const int tiles = ((nx + UM_BM - 1) / UM_BM) * ((ny + BN - 1) / BN);
    const int nkb = (int)(Kp / UM_BK);
    int splits = std::max(1, std::min(nkb, (148 + tiles - 1) / tiles));
    // at most UM_KB_CTA K blocks accumulate in FP32 per CTA; the partial
    // sums meet in FP64, so the rounding of the contraction stays near that
    // of one FP32 sum of UM_KB_CTA * 64 terms
    a.kb_per_cta = std::min((nkb + splits - 1) / splits, UM_KB_CTA);
    splits = (nkb + a.kb_per_cta - 1) / a.kb_per_cta;
    a.mode = 0;
    a.alpha = dV;
    a.S = S;
    a.lds = lds;
    a.err = err;
    return BN == 64 ? launch<64>(ta, tbm, a, splits, st) : launch<128>(ta, tbm, a, splits, st);
}

// Y (FP32, [npts][ldy], m columns) = alpha X C + beta Y, X FP32 [npts][ldx]
// (n columns), C FP64 [n][ldc].  Y must not alias X.
int umma_rowmul(const float *X, int64_t ldx, int n, const double *C, int64_t ldc, int m, float *Y, int64_t ldy,
                int64_t npts, double alpha, double beta, void *work, int *err, cudaStream_t st,
                UmmaSplitCache *xcache) {
    const int64_t Kp = round_up(n, UM_BK);
    const int BN = m <= 64 ? 64 : 128;
    const bool cached = xcache && xcache->buf;
    __nv_bfloat16 *PA = reinterpret_cast<__nv_bfloat16 *>(cached ? xcache->buf : work);
    __nv_bfloat16 *PB = cached ? reinterpret_cast<__nv_bfloat16 *>(work) : PA + 3 * round_up(npts, UM_BM) * Kp;
    if (!cache_hit(xcache, X, n, ldx, npts)) {
        k_split_n<float><<<2048, dim3(64, 4), 0, st>>>(X, ldx, (int)npts, n, (int)Kp, PA);
        cache_set(xcache, X, n, ldx, npts);
    }
    // C^T: rows = output columns, K = n
    dim3 tb(32, 8);
    k_split_t<double><<<dim3((unsigned)(Kp / 32), (unsigned)((m + 31) / 32)), tb, 0, st>>>(C, ldc, n, m, (int)Kp, PB);
    RS_LAUNCH_CHECK();
    CUtensorMap ta, tbm;
    RS_TRY(make_map(&ta, PA, (int)npts, (int)Kp, UM_BM));
    RS_TRY(make_map(&tbm, PB, m, (int)Kp, BN));
    UmmaArgs a{};
    a.M = (int)npts;
    a.N = m;
    a.K = (int)Kp;
    a.kb_per_cta = (int)(Kp / UM_BK);
    a.mode = 1;
    a.alpha = alpha;
    a.beta = beta;
    a.Y = Y;
    a.ldy = ldy;
    a.yvec = ((uintptr_t)Y % 16 == 0) && (ldy % 4 == 0);
    a.err = err;
    return BN == 64 ? launch<64>(ta, tbm, a, 1, st) : launch<128>(ta, tbm, a, 1, st);
}

}  // namespace rs

// ---------------------------------------------------------------- C ABI ---

using namespace rs;

extern "C" int64_t rs_tc_workspace_bytes(int64_t rows_a, int64_t rows_b, int64_t K) {
    if (rows_a < 1 || rows_b < 1 || K < 1) return -1;
    return umma_work_bytes(rows_a, rows_b, K) + 256;
}

static int tc_check(void *work, int64_t need_a, int64_t need_b, int64_t K, int **err, cudaStream_t st) {
    if (!work) return fail(RS_EINVAL, "tensor-core call: null workspace");
    *err = reinterpret_cast<int *>((char *)work + umma_work_bytes(need_a, need_b, K));
    RS_CUDA(cudaMemsetAsync(*err, 0, sizeof(int), st));
    return RS_OK;
}

static int tc_finish(int *err, cudaStream_t st) {
    int e = 0;
    RS_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    if (e) return fail(RS_ECUDA, "tensor-core pipeline wait timed out");
    return RS_OK;
}

extern "C" int rs_overlap_block_tc(const rs_grid *g, const float *X_dev, int64_t ldx, int nx, const float *Y_dev,
                                   int64_t ldy, int ny, double *S_dev, int64_t lds, void *work_dev, void *stream) {
    if (!g || !X_dev || !Y_dev || !S_dev) return fail(RS_EINVAL, "rs_overlap_block_tc: null argument");
    if (nx < 1 || ny < 1 || ldx < nx || ldy < ny || lds < ny) return fail(RS_EINVAL, "rs_overlap_block_tc: bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    int *err = nullptr;
    RS_TRY(tc_check(work_dev, nx, ny, g->npts, &err, st));
    RS_TRY(umma_gram(X_dev, ldx, nx, Y_dev, ldy, ny, g->npts, g->h * g->h * g->h, S_dev, lds, work_dev, err, st));
    return tc_finish(err, st);
}

extern "C" int rs_rotate_block(const float *X_dev, int64_t ldx, int n, const double *C_dev, int64_t ldc, int m,
                               float *Y_dev, int64_t ldy, int64_t npts, void *work_dev, void *stream) {
    if (!X_dev || !C_dev || !Y_dev) return fail(RS_EINVAL, "rs_rotate_block: null argument");
    if (n < 1 || m < 1 || npts < 1 || ldx < n || ldy < m || ldc < m) return fail(RS_EINVAL, "rs_rotate_block: bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    int *err = nullptr;
    RS_TRY(tc_check(work_dev, npts, m, n, &err, st));
    RS_TRY(umma_rowmul(X_dev, ldx, n, C_dev, ldc, m, Y_dev, ldy, npts, 1.0, 0.0, work_dev, err, st));
    return tc_finish(err, st);
}

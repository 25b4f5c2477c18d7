// Coarse 9-point block stencil on the 5th-generation tensor cores (row a8).
//
// y(X) = sum_{b=0..8} A_b(X) x(nbr_b(X)) with ncd x ncd complex blocks is, for
// every coarse site X, a real GEMM over the right-hand sides:
//   out[r][n] = sum_k xin[r][k] W_X[n][k],   M = RHS (tiles of 128),
//   N = 2 ncd (re/im interleaved outputs), K = 9 * 2 ncd (9 neighbour blocks),
// where xin[r] concatenates the 9 neighbours' complex vectors as interleaved
// (re, im) BF16 -- exactly the memory layout of a BF16 coarse field
// [rhs][Vc][ncd] complex -- and W_X is the real expansion of the blocks:
//   W[2i][2j] = Re A_ij, W[2i][2j+1] = -Im A_ij, W[2i+1][2j] = Im A_ij,
//   W[2i+1][2j+1] = Re A_ij.
// The output row is the FP32 coarse field [rhs][Vc][ncd] complex, directly.
//
// Kernel: one CTA (4 warps) per (X, RHS tile).  TMA brings 32-wide K chunks of
// xin (3D map over the coarse field: K, site, rhs; the neighbour index picks
// the site coordinate) and of W_X (2D map) into 64-byte-swizzled shared
// memory through a 4-stage mbarrier pipeline; thread 0 produces, thread 32
// issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M=128, N=2ncd, K=16)
// into a TMEM accumulator and releases each stage with tcgen05.commit; the 4
// warps then read their 32 TMEM lanes with tcgen05.ld and store FP32 rows.
// Every mbarrier wait is bounded: on timeout the kernel raises an error flag,
// skips the remaining work, lets the copies it issued land, frees its TMEM
// and returns; a producer wait also gives up as soon as another role of the
// CTA has failed.  The environment variable WD_TEST_TC_STALL=1 makes the MMA
// issuer wait, with a short limit, on a barrier nothing arrives on (a test of
// that failure path without any fault: the call returns WD_ETIMEOUT and the
// context stays usable).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "wd_internal.h"

namespace wd {

static constexpr int TC_M = 128;      // RHS per tile
static constexpr int TC_KC = 32;      // K elements (bf16) per chunk = one 64-byte swizzle row
static constexpr int TC_STAGES = 4;
static constexpr long TC_SPIN = 1L << 24;   // bounded waits
static constexpr long TC_SPIN_TEST = 1L << 10;   // the short limit of the stall test

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bounded wait for phase `parity` to complete; returns false after `limit`
// polls, or early once *abort (another role's failure flag) is set
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long limit = TC_SPIN,
                                          const volatile int *abort = nullptr) {
    const uint32_t a = smem_u32(bar);
    for (long i = 0; i < limit; ++i) {
        if (abort && (i & 255) == 255 && *abort) return false;
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1) : "memory");
}

// UMMA shared-memory descriptor, K-major operand with 64-byte swizzle:
// start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29, unused for
// swizzled K-major), stride byte offset >> 4 (32-45: 8-row groups, 512 B apart),
// descriptor version 1 (46-47), layout type 4 = SWIZZLE_64B (61-63).
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A BF16 (7-9 = 1),
// B BF16 (10-12 = 1), both K-major (15, 16 = 0), N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

struct TcArgs {
    const int *nbr;     // [Vc][9]
    float *y;           // FP32 coarse field [nrhs][Vc][ncd] complex
    int *err;           // set to a nonzero code on a timed-out wait
    int Vc, ncd, nrhs;
    int stall_test;     // 1: the MMA issuer waits (short limit) on a barrier nothing arrives on
};

// SPLIT: the blocks as two BF16 operands W + W_lo (mapw2) and the input as
// two BF16 fields x + x_lo (mapx2), multiplied into the same accumulator as
// W x + W_lo x + W x_lo (~16 significant bits of both operands; the product
// of the two remainders is below that)
template <int N, bool SPLIT>
__global__ void __launch_bounds__(128, 1) k_coarse_tc(const __grid_constant__ CUtensorMap mapx,
                                                      const __grid_constant__ CUtensorMap mapx2,
                                                      const __grid_constant__ CUtensorMap mapw,
                                                      const __grid_constant__ CUtensorMap mapw2, TcArgs A) {
    constexpr int KB = N / TC_KC;              // chunks per neighbour block (N = 2 ncd)
    constexpr int NCHUNK = 9 * KB;
    constexpr int NB = SPLIT ? 2 : 1;          // A and B operands per chunk
    constexpr uint32_t A1_BYTES = TC_M * TC_KC * 2, B1_BYTES = N * TC_KC * 2;
    constexpr uint32_t A_BYTES = NB * A1_BYTES, B_BYTES = NB * B1_BYTES;
    constexpr int TMEM_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned stage buffers (swizzle atoms must not straddle their base)
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = sA + TC_STAGES * A_BYTES;
    uint64_t *full = (uint64_t *)(sB + TC_STAGES * B_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *done = empty + TC_STAGES;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    volatile __shared__ int s_fail;
    __shared__ int s_issued[TC_STAGES];

    const int X = blockIdx.x / ((A.nrhs + TC_M - 1) / TC_M);
    const int r0 = (blockIdx.x % ((A.nrhs + TC_M - 1) / TC_M)) * TC_M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        s_fail = 0;
        for (int s = 0; s < TC_STAGES; ++s) s_issued[s] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        // producer: TMA loads of chunk kc into stage kc % S
        for (int kc = 0; kc < NCHUNK && !s_fail; ++kc) {
            const int s = kc % TC_STAGES;
            if (kc >= TC_STAGES && !mbar_wait(&empty[s], ((kc / TC_STAGES) - 1) & 1, TC_SPIN, &s_fail)) {
                if (!s_fail) s_fail = 1;
                break;
            }
            const int b = kc / KB, kk = (kc % KB) * TC_KC;
            const int nb = A.nbr[X * 9 + b];
            mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
            tma_load_3d(sA + s * A_BYTES, &mapx, &full[s], kk, nb, r0);
            tma_load_2d(sB + s * B_BYTES, &mapw, &full[s], kc * TC_KC, X * N);
            if (SPLIT) {
                tma_load_3d(sA + s * A_BYTES + A1_BYTES, &mapx2, &full[s], kk, nb, r0);
                tma_load_2d(sB + s * B_BYTES + B1_BYTES, &mapw2, &full[s], kc * TC_KC, X * N);
            }
            s_issued[s] += 1;
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16_f32(TC_M, N);
        for (int kc = 0; kc < NCHUNK; ++kc) {
            const int s = kc % TC_STAGES;
            const bool got = A.stall_test ? mbar_wait(done, 0, TC_SPIN_TEST) : mbar_wait(&full[s], (kc / TC_STAGES) & 1);
            if (!got) { s_fail = 2; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
            for (int k16 = 0; k16 < TC_KC / 16; ++k16)
#pragma unroll
                for (int q = 0; q < (SPLIT ? 3 : 1); ++q) {
                    // q = 0: W x, 1: W_lo x, 2: W x_lo
                    const uint64_t da = desc_sw64(a0 + (q == 2 ? A1_BYTES : 0) + 32 * k16);
                    const uint64_t db = desc_sw64(b0 + (q == 1 ? B1_BYTES : 0) + 32 * k16);
                    const uint32_t acc = (kc > 0 || k16 > 0 || q > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
            // release the stage when these MMAs have read it
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(done)) : "memory");
    }
    __syncwarp();
    // epilogue: all 4 warps wait for the accumulator, read their 32 lanes
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, A.stall_test ? TC_SPIN_TEST : TC_SPIN, &s_fail));
    if (!ok && lane == 0) s_fail = 3;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncwarp();
    const int r = r0 + warp * 32 + lane;
    float *out = A.y + ((size_t)r * A.Vc + X) * N;
    if (ok) {
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < A.nrhs) {
                float4 *o4 = (float4 *)(out + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    o4[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                        __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_fail && threadIdx.x == 0) {
        atomicExch(A.err, s_fail);
        // let the copies this CTA issued land before its shared memory is released:
        // the last load into stage s completes phase s_issued[s] - 1 of full[s]
        for (int s = 0; s < TC_STAGES; ++s)
            if (s_issued[s] > 0) mbar_wait(&full[s], (s_issued[s] - 1) & 1);
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// W_X[n][k] (bf16) from the FP64 blocks: [Vc][N = 2 ncd][K = 9 * 2 ncd], and
// (Wlo nullable) the rounding remainder bf16(v - W)
__global__ void k_build_w(const double2 *Dc, bf16 *W, bf16 *Wlo, int Vc, int ncd) {
    const long N = 2L * ncd, K = 18L * ncd;
    const long tot = (long)Vc * N * K;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const long k = e % K, n = (e / K) % N, X = e / (N * K);
        const int b = (int)(k / (2 * ncd)), j = (int)((k % (2 * ncd)) / 2), cin = (int)(k & 1);
        const int i = (int)(n / 2), cout = (int)(n & 1);
        const double2 a = Dc[(((size_t)X * 9 + b) * ncd + i) * ncd + j];
        double v;
        if (cout == 0) v = cin == 0 ? a.x : -a.y;
        else v = cin == 0 ? a.y : a.x;
        const bf16 hi = __double2bfloat16(v);
        W[e] = hi;
        if (Wlo) Wlo[e] = __double2bfloat16(v - (double)__bfloat162float(hi));
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static void *fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

static size_t tc_smem(int N, bool split) {
    return 1024 + TC_STAGES * (split ? 2 : 1) * ((size_t)TC_M * TC_KC * 2 + (size_t)N * TC_KC * 2) +
           (2 * TC_STAGES + 1) * 8 + 16;
}

// FP32 coarse field -> BF16 pair: hi = bf16(x), lo = bf16(x - hi)
__global__ void k_split_bf16(const float *x, bf16 *hi, bf16 *lo, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float v = x[i];
        const bf16 h = __float2bfloat16(v);
        hi[i] = h;
        lo[i] = __float2bfloat16(v - __bfloat162float(h));
    }
}

bool coarse_tc_ok(wd_ctx *c) { return c->mg && c->mg->Wtc != nullptr; }

int coarse_tc_build(wd_ctx *c) {
    wd_mg *g = c->mg;
    const int ncd = g->ncd;
    // tensor-core shapes: N = 2 ncd in {96, 192} (multiple of 32 for the 64-byte K chunks, <= 256)
    if (!((2 * ncd) % TC_KC == 0 && (2 * ncd == 96 || 2 * ncd == 192)) || !encode_fn()) return WD_OK;
    const size_t n = (size_t)g->Vc * 2 * ncd * 18 * ncd;
    if (cudaMalloc(&g->Wtc, n * sizeof(bf16)) != cudaSuccess) { cudaGetLastError(); g->Wtc = nullptr; return WD_OK; }
    if (cudaMalloc(&g->Wlo, n * sizeof(bf16)) != cudaSuccess) { cudaGetLastError(); g->Wlo = nullptr; }
    int *err;
    WD_TRY(ws_get(c, "tc.err", sizeof(int), (void **)&err));
    WD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->st));
    k_build_w<<<1184, 256, 0, c->st>>>(g->Dc, (bf16 *)g->Wtc, (bf16 *)g->Wlo, g->Vc, ncd);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int coarse_tc_apply(wd_ctx *c, const void *x_in, float *y, int nrhs, bool split) {
    wd_mg *g = c->mg;
    if (!g || !g->Wtc) { set_error("tensor-core coarse stencil unavailable"); return WD_ENOTSUP; }
    if (nrhs <= 0) return WD_OK;
    if (split && !g->Wlo) { set_error("tensor-core coarse stencil: no block remainders"); return WD_ENOTSUP; }
    const int N = 2 * g->ncd, K = 9 * N;
    // split: x_in is an FP32 field, split here into a BF16 pair
    const void *x_bf16 = x_in, *x_lo = x_in;
    if (split) {
        void *hi, *lo;
        const long n = (long)nrhs * g->Vc * N;
        WD_TRY(ws_get(c, "tc.xhi", (size_t)n * sizeof(bf16), &hi));
        WD_TRY(ws_get(c, "tc.xlo", (size_t)n * sizeof(bf16), &lo));
        k_split_bf16<<<1184, 256, 0, c->st>>>((const float *)x_in, (bf16 *)hi, (bf16 *)lo, n);
        c->launches++;
        x_bf16 = hi;
        x_lo = lo;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    CUtensorMap mx, mx2, mw, mw2;
    for (int q = 0; q < (split ? 2 : 1); ++q) {
        const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)g->Vc, (cuuint64_t)nrhs};
        const cuuint64_t strides[2] = {(cuuint64_t)N * 2, (cuuint64_t)g->Vc * N * 2};
        const cuuint32_t box[3] = {TC_KC, 1, TC_M};
        const cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(q ? &mx2 : &mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)(q ? x_lo : x_bf16), dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled (coarse field) failed: %d", (int)r); return WD_ECUDA; }
    }
    if (!split) mx2 = mx;
    {
        const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)g->Vc * N};
        const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
        const cuuint32_t box[2] = {TC_KC, (cuuint32_t)N};
        const cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g->Wtc, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled (blocks) failed: %d", (int)r); return WD_ECUDA; }
        mw2 = mw;
        if (split) {
            r = enc(&mw2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g->Wlo, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled (block remainders) failed: %d", (int)r); return WD_ECUDA; }
        }
    }
    int *err;
    WD_TRY(ws_get(c, "tc.err", sizeof(int), (void **)&err));
    TcArgs A;
    A.nbr = g->nbr; A.y = y; A.err = err; A.Vc = g->Vc; A.ncd = g->ncd; A.nrhs = nrhs;
    {
        const char *e = getenv("WD_TEST_TC_STALL");
        A.stall_test = e && atoi(e) == 1;
    }
    const unsigned grid = (unsigned)g->Vc * ((nrhs + TC_M - 1) / TC_M);
    const size_t smem = tc_smem(N, split);
    int slot;
    // algorithmic flops: 8 ncd^2 per block, 9 blocks, per site and RHS
    prof_begin(c, WD_K_COARSE, 8.0 * g->ncd * g->ncd * 9.0 * g->Vc * nrhs, &slot);
#define WD_TC_CASE(NN, SP)                                                                                 \
    if (N == NN && split == SP) {                                                                          \
        WD_CUDA(cudaFuncSetAttribute(k_coarse_tc<NN, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_coarse_tc<NN, SP><<<grid, 128, smem, c->st>>>(mx, mx2, mw, mw2, A);                              \
    }
    WD_TC_CASE(96, false) WD_TC_CASE(96, true) WD_TC_CASE(192, false) WD_TC_CASE(192, true)
#undef WD_TC_CASE
    prof_end(c, slot);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// nonzero if a tensor-core launch since the last reset timed out a wait
int coarse_tc_check(wd_ctx *c) {
    if (!c->mg || !c->mg->Wtc) return WD_OK;
    int *err;
    WD_TRY(ws_get(c, "tc.err", sizeof(int), (void **)&err));
    int h = 0;
    WD_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    if (h) {
        WD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->st));
        set_error("tensor-core coarse stencil: bounded wait gave up (code %d)", h);
        return WD_ETIMEOUT;
    }
    return WD_OK;
}

}  // namespace wd

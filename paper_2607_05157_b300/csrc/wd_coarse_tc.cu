// Coarse 9-point block stencil on the 5th-generation tensor cores.
//
// y(X) = sum_{b=0..8} A_b(X) x(nbr_b(X)) with ncd x ncd complex blocks is, for
// every coarse site X, two real GEMMs over the right-hand sides that share one
// compact block operand.  In 16-dof groups g (K = 16, one MMA deep):
//   D1 += Re x_g . B_g^T,  D2 += Im x_g . B_g^T,
//   B_g = [Re A_b(X)[:, g] ; Im A_b(X)[:, g]]   (N = 2 ncd rows),
// so D1 = [Re x Re A^T | Re x Im A^T], D2 = [Im x Re A^T | Im x Im A^T] and
//   Re y = D1[:, :ncd] - D2[:, ncd:],  Im y = D1[:, ncd:] + D2[:, :ncd].
// Neither operand is duplicated for the complex product: the blocks stream
// once at 4 bytes per complex entry (BF16), the input at the field's own size.
//
// Operand layout: every MMA tile is a run of 32-byte rows (16 BF16), stored in
// global memory as the image of its shared-memory tile under the 32-byte
// swizzle the MMA descriptors name (16-byte unit u of row r at u ^ ((r >> 2) & 1)),
// so that a stage is filled by plain bulk copies of whole tiles:
//   input  P: [Vc][G][RHS tile][Re|Im][rows][16], rows = 128 except in the
//             last tile (its RHS count rounded up to 8), so that one copy
//             brings the Re and the Im tile of a group;
//   blocks B: [Vc][9][G][2 ncd][16], tile (X, b, g) over the rows of B_g.
//
// Kernel: persistent, one CTA of 6 warps per SM, looping over the work items
// (X, RHS tile of 128).  Warp 0 (one lane) produces: bulk copies
// (cp.async.bulk, completion counted on the stage's mbarrier) of TC_CPS groups
// per stage into a ring that runs on across items.  Warp 1 allocates TMEM and
// (one lane) issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
// N = 2 ncd) into one of two accumulator sets, releasing each stage with
// tcgen05.commit and handing a finished set to the epilogue with another.
// Warps 2-5 drain a set (tcgen05.ld of their 32 TMEM lanes each), give it back
// and store interleaved FP32 complex rows while the next item's MMAs run.
// With BF16 pairs (three MMAs per product, MMA-bound) a tile of at most 64
// RHS is stacked: its Re and Im rows lie back to back inside one 128-row
// operand, one MMA gives D1 in the first lanes and D2 right after them, and
// the epilogue warps pass the D2 rows through shared memory to the lanes of
// their RHS (half the MMAs; 64 RHS on 24^3x48: 0.132 -> 0.119 ms).  The
// epilogue warps agree on each accumulator wait's outcome before any barrier
// among them, so a timeout ends all four together.
// Every mbarrier wait is bounded: on timeout the kernel raises an error flag,
// all roles stop, the copies and MMAs already issued complete, the TMEM is
// freed and the kernel returns.  The environment variable WD_TEST_TC_STALL=1
// makes the MMA issuer wait, with a short limit, on a barrier nothing arrives
// on (a test of that failure path without any fault: the call returns
// WD_ETIMEOUT and the context stays usable).
#include "wd_internal.h"

namespace wd {

static constexpr int TC_M = 128;      // RHS per tile
static constexpr int TC_KC = 16;      // K elements (bf16) per tile row = one 32-byte swizzle row
static constexpr int TC_MAXSTAGES = 8;
static constexpr int TC_THREADS = 192;   // producer warp, MMA warp, 4 epilogue warps
static constexpr int TC_CPS = 3;         // 16-dof groups per stage (one neighbour block at ncd = 48)
// ring depth: 165-200 KB of stages for the one CTA per SM
__host__ __device__ constexpr int tc_stages(int NC, bool split) {
    return NC <= 48 ? (split ? 3 : 5) : (split ? 2 : 4);
}
static constexpr long TC_SPIN = 1L << 24;   // bounded waits
static constexpr long TC_SPIN_TEST = 1L << 10;   // the short limit of the stall test

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, counted on the mbarrier's transaction count
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// UMMA shared-memory descriptor, K-major operand with 32-byte swizzle:
// start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29, unused for
// swizzled K-major), stride byte offset >> 4 (32-45: 8-row groups, 256 B apart),
// descriptor version 1 (46-47), layout type 6 = SWIZZLE_32B (61-63).
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A BF16 (7-9 = 1),
// B BF16 (10-12 = 1), both K-major (15, 16 = 0), N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 16 consecutive TMEM columns of this warp's 32 lanes (one 32-bit value each)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

struct TcArgs {
    const bf16 *P, *Plo;   // input operand (and remainder; Plo = P when not split)
    const bf16 *B, *Blo;   // block operand (and remainder)
    const int *nbr;     // [Vc][9]
    float *y;           // FP32 coarse field [nrhs][Vc][ncd] complex
    int *err;           // set to a nonzero code on a timed-out wait
    int Vc, ncd, nrhs;
    int nitems;         // Vc x RHS tiles, handed out round-robin over the CTAs
    int nrhs8;          // nrhs rounded up to 8: the rows of one (site, group) of P
    int stall_test;     // 1: the MMA issuer waits (short limit) on a barrier nothing arrives on
};

// SPLIT: the blocks and the input as BF16 pairs (hi + lo: B, B_lo and P,
// P_lo), multiplied into the same accumulators as B P + B_lo P + B P_lo (~16
// significant bits of both operands; the product of the two remainders is
// below that).  NC = ncd; the MMA's N is 2 NC.
template <int NC, bool SPLIT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_coarse_tc(TcArgs A) {
    constexpr int S = tc_stages(NC, SPLIT);
    constexpr int G = NC / 16;                 // 16-dof groups per block
    constexpr int NGRP = 9 * G;                // groups per item
    constexpr int NSTEP = NGRP / TC_CPS;       // stages per item
    constexpr int NQ = SPLIT ? 2 : 1;          // hi (, lo) tiles of each operand
    constexpr int N = 2 * NC;
    // a stage: input groups [NQ][TC_CPS] of GA bytes (128 Re rows, then 128
    // Im rows of 32 bytes), then block tiles [NQ][TC_CPS]
    constexpr uint32_t GA = 2 * TC_M * TC_KC * 2, B1_BYTES = N * TC_KC * 2;
    constexpr uint32_t A_BYTES = NQ * TC_CPS * GA, B_BYTES = NQ * TC_CPS * B1_BYTES;
    constexpr uint32_t DOFF = N <= 128 ? 128 : 256;   // TMEM columns of D1, then D2
    constexpr int NSET = 4 * DOFF <= 512 ? 2 : 1;     // accumulator sets (double buffer when they fit)
    constexpr int TMEM_COLS = 512;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned stage buffers (swizzle atoms must not straddle their base)
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = sA + S * A_BYTES;
    uint64_t *full = (uint64_t *)(sB + S * B_BYTES);
    uint64_t *empty = full + S;
    uint64_t *tfull = empty + S;               // [NSET] accumulator set ready (MMA -> epilogue)
    uint64_t *tempty = tfull + 2;              // [NSET] accumulator set drained (epilogue -> MMA)
    uint64_t *drain = tempty + 2;              // the MMA issuer's last commit
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    // [TC_M / 2][32] Im-input rows of a stacked tile, 16-byte aligned for float4
    float *xch = (float *)(((uintptr_t)(tmem_slot + 1) + 15) & ~(uintptr_t)15);
    volatile __shared__ int s_fail;
    __shared__ int s_issued[TC_MAXSTAGES];
    __shared__ int s_epi_ok[2][4];             // epilogue warps' view of an item's accumulator wait

    const int ntile = (A.nrhs + TC_M - 1) / TC_M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int t = 0; t < 2; ++t) { mbar_init(&tfull[t], 1); mbar_init(&tempty[t], 4); }
        mbar_init(drain, 1);
        s_fail = 0;
        for (int s = 0; s < S; ++s) s_issued[s] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        // producer: bulk copies of TC_CPS groups per stage fill into stage
        // gs % S.  An input tile holds the item's rows of RHS (fewer than 128
        // in the last tile); the MMA still reads 128 rows: the rows past them
        // hold stale data and give accumulator rows that are never stored.
        // The 9 neighbour indices of the next item are loaded while this one
        // is issued, so that no copy waits on a dependent global load.
        uint32_t gs = 0;                       // stage fills, counted over all items
        int nbv[9], nbn[9];
        if (blockIdx.x < A.nitems) {
#pragma unroll
            for (int b = 0; b < 9; ++b) nbv[b] = A.nbr[(blockIdx.x / ntile) * 9 + b];
        }
        for (int it = blockIdx.x; it < A.nitems && !s_fail; it += gridDim.x) {
            const int X = it / ntile, r0 = (it % ntile) * TC_M;
            const int itn = it + gridDim.x;
            if (itn < A.nitems) {
#pragma unroll
                for (int b = 0; b < 9; ++b) nbn[b] = A.nbr[(itn / ntile) * 9 + b];
            }
            // rows of this tile in P (a multiple of 8); its Im half follows its Re half
            const int rows = min(TC_M, A.nrhs8 - r0);
            const uint32_t abytes = 2u * (uint32_t)rows * TC_KC * 2;
            const uint32_t tx = NQ * TC_CPS * (abytes + B1_BYTES);
            const size_t bx = (size_t)X * NGRP * N * TC_KC;
            bool stop = false;
            for (int st = 0; st < NSTEP; ++st, ++gs) {
                const int s = (int)(gs % S);
                if (gs >= S && !mbar_wait(&empty[s], ((gs / S) - 1) & 1, TC_SPIN, &s_fail)) {
                    if (!s_fail) s_fail = 1;
                    stop = true;
                    break;
                }
                unsigned char *a = sA + s * A_BYTES;
                unsigned char *bb = sB + s * B_BYTES;
                mbar_expect_tx(&full[s], tx);
                // the stage's TC_CPS block tiles are consecutive in B
                const size_t bo = bx + (size_t)st * TC_CPS * N * TC_KC;
                bulk_load(bb, A.B + bo, TC_CPS * B1_BYTES, &full[s]);
                if (SPLIT) bulk_load(bb + TC_CPS * B1_BYTES, A.Blo + bo, TC_CPS * B1_BYTES, &full[s]);
#pragma unroll
                for (int c = 0; c < TC_CPS; ++c) {
                    const int kg = st * TC_CPS + c, b = kg / G, g = kg % G;
                    int nb = nbv[0];
#pragma unroll
                    for (int q = 1; q < 9; ++q) nb = b == q ? nbv[q] : nb;
                    const size_t ao = (((size_t)nb * G + g) * A.nrhs8 + r0) * 2 * TC_KC;
                    bulk_load(a + c * GA, A.P + ao, abytes, &full[s]);
                    if (SPLIT) bulk_load(a + (TC_CPS + c) * GA, A.Plo + ao, abytes, &full[s]);
                }
                s_issued[s] += 1;
            }
            if (stop) break;
#pragma unroll
            for (int b = 0; b < 9; ++b) nbv[b] = nbn[b];
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer: per group, D1 += Re x . B^T and D2 += Im x . B^T
        constexpr uint32_t idesc = idesc_bf16_f32(TC_M, N);
        // descriptors of stage 0; a stage's, and a tile's within it, differ
        // only by a constant added to the 14-bit start-address field
        const uint64_t dA0 = desc_sw32(smem_u32(sA)), dB0 = desc_sw32(smem_u32(sB));
        uint32_t gs = 0;
        int li = 0;
        if (A.stall_test && !mbar_wait(drain, 0, TC_SPIN_TEST)) s_fail = 2;
        for (int it = blockIdx.x; it < A.nitems && !s_fail; it += gridDim.x, ++li) {
            const int set = li % NSET, use = li / NSET;
            if (use > 0 && !mbar_wait(&tempty[set], (uint32_t)(use - 1) & 1, TC_SPIN, &s_fail)) {
                if (!s_fail) s_fail = 2;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t dcol = tmem + (uint32_t)set * 2 * DOFF;
            // the Im tile of a group starts `rows` rows after its Re tile (a
            // multiple of 8 rows, so on a swizzle-atom boundary); the MMA reads
            // 128 rows from either start, all inside the group's 2 x 128 rows
            const int rows_it = min(TC_M, A.nrhs8 - (it % ntile) * TC_M);
            const uint32_t imoff = (uint32_t)rows_it * TC_KC * 2;
            // a tile of at most TC_M / 2 rows is stacked: its Re rows and then its
            // Im rows are the first 2 rows_it of one 128-row operand, so the
            // MMA from the Re start alone gives both products (accumulator
            // lanes < rows_it: Re x B^T, rows_it .. 2 rows_it - 1: Im x B^T).
            // Half the MMAs: it pays where they bind (BF16 pairs, three MMAs
            // per product), not where the copies do (BF16)
            const bool stacked = SPLIT && 2 * rows_it <= TC_M;
            bool ok = true;
            for (int st = 0; st < NSTEP; ++st, ++gs) {
                const int s = (int)(gs % S);
                if (!mbar_wait(&full[s], (gs / S) & 1, TC_SPIN, &s_fail)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint64_t dA = dA0 + (uint64_t)(s * (A_BYTES >> 4)), dB = dB0 + (uint64_t)(s * (B_BYTES >> 4));
                const uint32_t later = st > 0 ? 1u : 0u;
#pragma unroll
                for (int c = 0; c < TC_CPS; ++c)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int q = 0; q < (SPLIT ? 3 : 1); ++q) {
                            if (h == 1 && stacked) continue;
                            // q = 0: P B, 1: P B_lo, 2: P_lo B
                            const uint32_t ao = ((q == 2 ? TC_CPS : 0) + c) * GA + (h ? imoff : 0u);
                            const uint32_t bo = ((q == 1 ? TC_CPS : 0) + c) * B1_BYTES;
                            // the first MMA into each accumulator of an item overwrites it
                            const uint32_t acc = (c > 0 || q > 0) ? 1u : later;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                ::"r"(dcol + (uint32_t)h * DOFF), "l"(dA + (ao >> 4)), "l"(dB + (bo >> 4)), "r"(idesc),
                                  "r"(acc));
                        }
                // release the stage when these MMAs have read it
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(&empty[s])) : "memory");
            }
            if (!ok) { if (!s_fail) s_fail = 2; break; }
            // the set is complete once these MMAs are
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&tfull[set])) : "memory");
        }
        // every MMA issued has completed before the CTA may free TMEM or shared memory
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(drain)) : "memory");
        if (!mbar_wait(drain, 0) && !s_fail) s_fail = 4;
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the lanes its
        // position in the warpgroup may access), i.e. RHS rows r0 + 32 (w % 4) + lane
        const int quarter = warp & 3;
        int li = 0;
        for (int it = blockIdx.x; it < A.nitems; it += gridDim.x, ++li) {
            const int set = li % NSET, use = li / NSET;
            const bool got = __all_sync(0xffffffffu, mbar_wait(&tfull[set], (uint32_t)use & 1, TC_SPIN, &s_fail));
            // the four epilogue warps agree on the outcome before any barrier
            // among them (flags double-buffered by item parity: a warp rewrites
            // a buffer only after the next item's vote, which every warp reaches
            // after reading it)
            if (lane == 0) s_epi_ok[li & 1][quarter] = got ? 1 : 0;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const bool all_ok = s_epi_ok[li & 1][0] && s_epi_ok[li & 1][1] && s_epi_ok[li & 1][2] && s_epi_ok[li & 1][3];
            if (!all_ok) { if (lane == 0 && !got && !s_fail) s_fail = 3; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int rows_it = min(TC_M, A.nrhs8 - (it % ntile) * TC_M);
            const int L = quarter * 32 + lane;                   // the accumulator lane this thread reads
            const int X = it / ntile, r = (it % ntile) * TC_M + L;
            float *out = A.y + ((size_t)r * A.Vc + X) * 2 * NC;
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)set * 2 * DOFF;
            if (SPLIT && 2 * rows_it <= TC_M) {
                // stacked tile: lanes rows_it .. 2 rows_it - 1 hold the Im x B^T rows;
                // they pass them through shared memory to the lanes of their RHS
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += 16) {
                    uint32_t u[16], v[16];
                    tmem_ld16(tbase + (uint32_t)c0, u);
                    tmem_ld16(tbase + (uint32_t)(NC + c0), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (L >= rows_it && L < 2 * rows_it) {
                        float4 *x4 = (float4 *)(xch + (size_t)(L - rows_it) * 32);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            x4[q] = make_float4(__uint_as_float(u[4 * q]), __uint_as_float(u[4 * q + 1]),
                                                __uint_as_float(u[4 * q + 2]), __uint_as_float(u[4 * q + 3]));
                            x4[4 + q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                                    __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                        }
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    if (L < rows_it && r < A.nrhs) {
                        // u = Re x Re A, v = Re x Im A (own lane), w = Im x Re A, z = Im x Im A
                        const float *wz = xch + (size_t)L * 32;
                        float4 *o4 = (float4 *)(out + 2 * c0);
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            o4[q] = make_float4(__uint_as_float(u[2 * q]) - wz[16 + 2 * q],
                                                __uint_as_float(v[2 * q]) + wz[2 * q],
                                                __uint_as_float(u[2 * q + 1]) - wz[16 + 2 * q + 1],
                                                __uint_as_float(v[2 * q + 1]) + wz[2 * q + 1]);
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                }
            } else {
#pragma unroll
            for (int c0 = 0; c0 < NC; c0 += 16) {
                // u = Re x Re A, v = Re x Im A, w = Im x Re A, z = Im x Im A (16 columns each)
                uint32_t u[16], v[16], w[16], z[16];
                tmem_ld16(tbase + (uint32_t)c0, u);
                tmem_ld16(tbase + (uint32_t)(NC + c0), v);
                tmem_ld16(tbase + DOFF + (uint32_t)c0, w);
                tmem_ld16(tbase + DOFF + (uint32_t)(NC + c0), z);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (r < A.nrhs) {
                    float4 *o4 = (float4 *)(out + 2 * c0);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        o4[q] = make_float4(__uint_as_float(u[2 * q]) - __uint_as_float(z[2 * q]),
                                            __uint_as_float(v[2 * q]) + __uint_as_float(w[2 * q]),
                                            __uint_as_float(u[2 * q + 1]) - __uint_as_float(z[2 * q + 1]),
                                            __uint_as_float(v[2 * q + 1]) + __uint_as_float(w[2 * q + 1]));
                }
            }
            }
            // hand the set back to the MMA issuer
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[set]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_fail && threadIdx.x == 0) {
        atomicExch(A.err, s_fail);
        // let the copies this CTA issued land before its shared memory is released:
        // the last fill of stage s completes phase s_issued[s] - 1 of full[s]
        for (int s = 0; s < S; ++s)
            if (s_issued[s] > 0) mbar_wait(&full[s], (s_issued[s] - 1) & 1);
    }
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// position of entry t (0..15) of row r in a 32-byte-swizzled tile of 32-byte
// rows: the 16-byte unit t / 8 moves to unit (t / 8) ^ ((r >> 2) & 1)
__device__ __forceinline__ int sw32(int r, int t) { return r * 16 + ((((t >> 3) ^ (r >> 2)) & 1) << 3) + (t & 7); }

// The block operand B (bf16) from the FP64 blocks: [Vc][9][G][2 ncd][16] in
// the tile image; tile (X, b, g), row n, entry t: Re A_b[n][16 g + t] for
// n < ncd, Im A_b[n - ncd][16 g + t] beyond; and (Blo nullable) the rounding
// remainders bf16(v - B)
__global__ void k_build_b(const double2 *Dc, bf16 *B, bf16 *Blo, int Vc, int ncd) {
    const int G = ncd / 16, N = 2 * ncd;
    const long tot = (long)Vc * 9 * G * N * 16;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e & 15);
        const long row = e >> 4;
        const int n = (int)(row % N);
        const long tile = row / N;                           // (X, b, g)
        const int g = (int)(tile % G), b = (int)((tile / G) % 9);
        const long X = tile / (9 * G);
        const int i = n < ncd ? n : n - ncd, j = g * 16 + t;
        const double2 a = Dc[(((size_t)X * 9 + b) * ncd + i) * ncd + j];
        const double v = n < ncd ? a.x : a.y;
        const bf16 hi = __double2bfloat16(v);
        const size_t o = (size_t)tile * N * 16 + sw32(n, t);
        B[o] = hi;
        if (Blo) Blo[o] = __double2bfloat16(v - (double)__bfloat162float(hi));
    }
}

// FP32 coarse field [rhs][Vc][ncd] complex -> the input operand P (bf16) in
// the tile image: per site and 16-dof group, per RHS tile of 128 (the last
// one's rows rounded up to 8), the Re tile and then the Im tile of its rows;
// and (lo nullable) the rounding remainders.  Rows past nrhs stay unwritten.
__global__ void k_to_planar(const float2 *x, bf16 *p, bf16 *plo, int nrhs, int Vc, int ncd) {
    const long n = (long)nrhs * Vc * ncd;
    const int G = ncd / 16, nrhs8 = (nrhs + 7) & ~7;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e % ncd);
        const long v = (e / ncd) % Vc;
        const int r = (int)(e / ((long)ncd * Vc));
        const int r0 = r & ~(TC_M - 1), rows = min(TC_M, nrhs8 - r0);
        const float2 z = x[e];
        const size_t tre = (((size_t)v * G + (j >> 4)) * nrhs8 + r0) * 2 * 16;
        const size_t ore = tre + sw32(r - r0, j & 15), oim = ore + (size_t)rows * 16;
        const bf16 re = __float2bfloat16(z.x), im = __float2bfloat16(z.y);
        p[ore] = re;
        p[oim] = im;
        if (plo) {
            plo[ore] = __float2bfloat16(z.x - __bfloat162float(re));
            plo[oim] = __float2bfloat16(z.y - __bfloat162float(im));
        }
    }
}

// the epilogue's exchange of the Im-input rows of stacked tiles (below): up to
// TC_M / 2 rows x 32 FP32 values of one 16-column chunk
static constexpr size_t TC_XCH_BYTES = (size_t)(TC_M / 2) * 32 * 4;

static size_t tc_smem(int NC, bool split) {
    const size_t q = split ? 2 : 1;
    const int S = tc_stages(NC, split);
    return 1024 + S * q * TC_CPS * (2 * (size_t)TC_M * TC_KC * 2 + (size_t)2 * NC * TC_KC * 2) + (2 * S + 5) * 8 + 32 +
           TC_XCH_BYTES;
}

bool coarse_tc_ok(wd_ctx *c) { return c->mg && c->mg->Wtc != nullptr; }

int coarse_tc_build(wd_ctx *c) {
    wd_mg *g = c->mg;
    const int ncd = g->ncd;
    // tensor-core shapes: ncd in {48, 96} (16-dof groups, MMA N = 2 ncd <= 256)
    if (!(ncd == 48 || ncd == 96)) return WD_OK;
    const size_t n = (size_t)g->Vc * ncd * 18 * ncd;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&g->tc_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g->tc_sms <= 0)
        g->tc_sms = 148;
    // (kept from a previous setup of the same geometry, else allocated)
    if (!g->Wtc && cudaMalloc(&g->Wtc, n * sizeof(bf16)) != cudaSuccess) { cudaGetLastError(); g->Wtc = nullptr; return WD_OK; }
    if (!g->Wlo && cudaMalloc(&g->Wlo, n * sizeof(bf16)) != cudaSuccess) { cudaGetLastError(); g->Wlo = nullptr; }
    int *err;
    WD_TRY(ws_get(c, "tc.err", sizeof(int), (void **)&err));
    WD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->st));
    k_build_b<<<1184, 256, 0, c->st>>>(g->Dc, (bf16 *)g->Wtc, (bf16 *)g->Wlo, g->Vc, ncd);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int coarse_tc_apply(wd_ctx *c, const void *x_in, float *y, int nrhs, bool split) {
    wd_mg *g = c->mg;
    if (!g || !g->Wtc) { set_error("tensor-core coarse stencil unavailable"); return WD_ENOTSUP; }
    if (nrhs <= 0) return WD_OK;
    if (split && !g->Wlo) { set_error("tensor-core coarse stencil: no block remainders"); return WD_ENOTSUP; }
    const int NC = g->ncd;
    // the planar BF16 input (and its remainders when split)
    void *pl[2] = {nullptr, nullptr};
    const int nrhs8 = (nrhs + 7) & ~7;
    const long nel = (long)nrhs8 * g->Vc * 2 * NC;
    WD_TRY(ws_get(c, "tc.p", (size_t)nel * sizeof(bf16), &pl[0]));
    if (split) WD_TRY(ws_get(c, "tc.plo", (size_t)nel * sizeof(bf16), &pl[1]));
    k_to_planar<<<1184, 256, 0, c->st>>>((const float2 *)x_in, (bf16 *)pl[0], (bf16 *)pl[1], nrhs, g->Vc, NC);
    c->launches++;
    int *err;
    WD_TRY(ws_get(c, "tc.err", sizeof(int), (void **)&err));
    TcArgs A;
    A.nbr = g->nbr; A.y = y; A.err = err; A.Vc = g->Vc; A.ncd = g->ncd; A.nrhs = nrhs;
    A.P = (const bf16 *)pl[0]; A.Plo = split ? (const bf16 *)pl[1] : A.P;
    A.B = (const bf16 *)g->Wtc; A.Blo = split ? (const bf16 *)g->Wlo : A.B;
    A.nitems = g->Vc * ((nrhs + TC_M - 1) / TC_M);
    A.nrhs8 = nrhs8;
    {
        const char *e = getenv("WD_TEST_TC_STALL");
        A.stall_test = e && atoi(e) == 1;
    }
    const unsigned grid = (unsigned)std::min(A.nitems, g->tc_sms);
    const size_t smem = tc_smem(NC, split);
    int slot;
    // algorithmic flops: 8 ncd^2 per block, 9 blocks, per site and RHS
    prof_begin(c, WD_K_COARSE, 8.0 * g->ncd * g->ncd * 9.0 * g->Vc * nrhs, &slot);
#define WD_TC_CASE(NN, SP)                                                                                 \
    if (NC == NN && split == SP) {                                                                         \
        WD_CUDA(cudaFuncSetAttribute(k_coarse_tc<NN, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_coarse_tc<NN, SP><<<grid, TC_THREADS, smem, c->st>>>(A);          \
    }
    WD_TC_CASE(48, false) WD_TC_CASE(48, true) WD_TC_CASE(96, false) WD_TC_CASE(96, true)
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

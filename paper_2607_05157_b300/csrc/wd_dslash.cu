// Fine Wilson hopping stencil on one parity, many right-hand sides.
//
// (H psi)(x) = sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)]
// (the hopping part of the Wilson-Dirac operator; the paper, Sec. 1, fixes D
// only as nearest-neighbour 12x12 blocks on a 4D torus -- the standard
// hopping form is the reading used throughout).
//
// One thread owns one output site and a tile of R right-hand sides.  For each
// of the 8 directions it loads the link once (9 complex) and applies it to the
// spin-projected half-spinors of all R RHS, so each link is read once per
// R-tile; consecutive CTAs cover the RHS tiles of the same site block, so the
// other tiles find the links in L2.  The spin projection halves the SU(3)
// work: (1 -/+ g_mu) psi has rank 2 in the chiral basis, g_mu = [[0,A],[A^dag,0]]:
//   h = psi_up + sign*A psi_down,  lower half = sign*A^dag (U h).
// Epilogue: out = a*w + c*w2 + b*(H in), w/w2 same-parity fields (nullable).
#include <type_traits>

#include "wd_internal.h"
#include "wd_spin.cuh"

namespace wd {

// out[i] = sum_j u[3i+j] in[j] for both half-spinor spins
template <typename R>
__device__ __forceinline__ void su3_mul(const cx<R> u[9], const cx<R> in[6], cx<R> out[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cx<R> a = cmake(R(0), R(0));
#pragma unroll
            for (int j = 0; j < 3; ++j) cfma(a, u[3 * i + j], in[3 * s + j]);
            out[3 * s + i] = a;
        }
}

template <typename SIn, typename G, int R, int D, bool DAG, typename RT>
__device__ __forceinline__ void hop_dir(const HopArgs &A, int s, int nb, int rb, cx<RT> acc[][12]) {
    constexpr int MU = D & 3;
    constexpr bool FWD = D < 4;
    // D uses (1 - g) forward and (1 + g) backward; D^dag swaps them.
    constexpr int SIGN = (FWD != DAG) ? -1 : +1;
    const long Vh = A.g.Vh;
    cx<RT> u[9];
    LIO<G>::load((const char *)A.gauge + (size_t)D * 9 * Vh * LIO<G>::ELEM, Vh, s, u);
    constexpr int NCH = SIO<SIn>::NCH;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = tile_rhs(A, rb, r, R);
        if (rhs >= 0) {
            cx<RT> psi[12], h[6], uh[6];
            SIO<SIn>::load((const uint4 *)A.in + (size_t)rhs * NCH * Vh, Vh, nb, psi);
            spin_project<MU, SIGN>(psi, h);
            su3_mul(u, h, uh);
            spin_reconstruct_add<MU, SIGN>(acc[r], uh);
        }
    }
}

template <typename SIn, typename SOut, typename SW, typename G, int R, bool DAG>
__global__ void __launch_bounds__(256) hop_kernel(HopArgs A) {
    typedef typename RealOf<SIn>::type RT;
    const int rb = blockIdx.x % A.nrb;
    const int s = (blockIdx.x / A.nrb) * blockDim.x + threadIdx.x;
    if (s >= A.g.Vh || tile_rhs(A, rb, 0, R) < 0) return;   // no site, or a tile with no working RHS
    const Geom &g = A.g;
    int x, y, z, t;
    eo_coords(g, A.p, s, x, y, z, t);
    const int xp = x + 1 == g.X ? 0 : x + 1, xm = x == 0 ? g.X - 1 : x - 1;
    const int yp = y + 1 == g.Y ? 0 : y + 1, ym = y == 0 ? g.Y - 1 : y - 1;
    const int zp = z + 1 == g.Z ? 0 : z + 1, zm = z == 0 ? g.Z - 1 : z - 1;
    const int tp = t + 1 == g.T ? 0 : t + 1, tm = t == 0 ? g.T - 1 : t - 1;

    cx<RT> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = cmake(RT(0), RT(0));

    hop_dir<SIn, G, R, 0, DAG>(A, s, eo_index(g, xp, y, z, t), rb, acc);
    hop_dir<SIn, G, R, 1, DAG>(A, s, eo_index(g, x, yp, z, t), rb, acc);
    hop_dir<SIn, G, R, 2, DAG>(A, s, eo_index(g, x, y, zp, t), rb, acc);
    hop_dir<SIn, G, R, 3, DAG>(A, s, eo_index(g, x, y, z, tp), rb, acc);
    hop_dir<SIn, G, R, 4, DAG>(A, s, eo_index(g, xm, y, z, t), rb, acc);
    hop_dir<SIn, G, R, 5, DAG>(A, s, eo_index(g, x, ym, z, t), rb, acc);
    hop_dir<SIn, G, R, 6, DAG>(A, s, eo_index(g, x, y, zm, t), rb, acc);
    hop_dir<SIn, G, R, 7, DAG>(A, s, eo_index(g, x, y, z, tm), rb, acc);

    const long Vh = g.Vh;
    constexpr int NO = SIO<SOut>::NCH, NW = SIO<SW>::NCH;
    const RT a = (RT)A.a, b = (RT)A.b, c = (RT)A.c;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = tile_rhs(A, rb, r, R);
        if (rhs < 0) break;
        cx<RT> o[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = b * acc[r][k];
        if (A.w) {
            cx<RT> wv[12];
            SIO<SW>::load((const uint4 *)A.w + (size_t)rhs * NW * Vh, Vh, s, wv);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = o[k] + a * wv[k];
        }
        if (A.w2) {
            cx<RT> wv[12];
            SIO<SW>::load((const uint4 *)A.w2 + (size_t)rhs * NW * Vh, Vh, s, wv);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = o[k] + c * wv[k];
        }
        SIO<SOut>::store((uint4 *)A.out + (size_t)rhs * NO * Vh, Vh, s, o);
    }
}

// ---- FP32 arithmetic on packed pairs (Blackwell f32x2 FMA/ADD) -------------
// Complex numbers are float2 (re, im).  A complex multiply-add u*h + acc is two
// packed FMAs: (u.re, u.re) * (h.re, h.im) + acc, then (-u.im, u.im) * (h.im, h.re);
// the broadcast / sign pairs of a link are built once and reused by both
// half-spinor spins and every RHS of the tile, the swapped h once per h.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sw(float2 a) { return make_float2(a.y, a.x); }

template <int MU, int SIGN>
__device__ __forceinline__ void proj_f2(const float2 p[12], float2 h[6]) {
    const float S = (float)SIGN;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        if (MU == 0) {        // A = -i s1: (A pd) = (-i p3, -i p2); -i q = (q.im, -q.re)
            h[c] = __ffma2_rn(sw(p3), f2(S, -S), p0);
            h[3 + c] = __ffma2_rn(sw(p2), f2(S, -S), p1);
        } else if (MU == 1) { // A = -i s2: (-p3, p2)
            h[c] = __ffma2_rn(p3, f2(-S, -S), p0);
            h[3 + c] = __ffma2_rn(p2, f2(S, S), p1);
        } else if (MU == 2) { // A = -i s3: (-i p2, i p3); i q = (-q.im, q.re)
            h[c] = __ffma2_rn(sw(p2), f2(S, -S), p0);
            h[3 + c] = __ffma2_rn(sw(p3), f2(-S, S), p1);
        } else {              // A = 1
            h[c] = __ffma2_rn(p2, f2(S, S), p0);
            h[3 + c] = __ffma2_rn(p3, f2(S, S), p1);
        }
    }
}

template <int MU, int SIGN>
__device__ __forceinline__ void recon_f2(float2 acc[12], const float2 h[6]) {
    const float S = (float)SIGN;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 h0 = h[c], h1 = h[3 + c];
        acc[c] = __fadd2_rn(acc[c], h0);
        acc[3 + c] = __fadd2_rn(acc[3 + c], h1);
        if (MU == 0) {        // A^dag (h0, h1) = (i h1, i h0)
            acc[6 + c] = __ffma2_rn(sw(h1), f2(-S, S), acc[6 + c]);
            acc[9 + c] = __ffma2_rn(sw(h0), f2(-S, S), acc[9 + c]);
        } else if (MU == 1) { // (h1, -h0)
            acc[6 + c] = __ffma2_rn(h1, f2(S, S), acc[6 + c]);
            acc[9 + c] = __ffma2_rn(h0, f2(-S, -S), acc[9 + c]);
        } else if (MU == 2) { // (i h0, -i h1)
            acc[6 + c] = __ffma2_rn(sw(h0), f2(-S, S), acc[6 + c]);
            acc[9 + c] = __ffma2_rn(sw(h1), f2(S, -S), acc[9 + c]);
        } else {              // (h0, h1)
            acc[6 + c] = __ffma2_rn(h0, f2(S, S), acc[6 + c]);
            acc[9 + c] = __ffma2_rn(h1, f2(S, S), acc[9 + c]);
        }
    }
}

template <typename S> __device__ __forceinline__ void load_f2(const void *p, long Vh, long s, float2 v[12]) {
    cx<float> t[12];
    SIO<S>::load(p, Vh, s, t);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = make_float2(t[k].re, t[k].im);
}

// Prefetch of the next direction's link and neighbour spinors (PF = 1: into
// L1, PF = 2: into L2): the loads of direction d+1 are in flight while
// direction d computes, without holding registers for them.
template <int PF> __device__ __forceinline__ void prefetch_line(const void *p) {
    if constexpr (PF == 1) asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    else if constexpr (PF == 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <typename SIn, typename G, int R, int D, int PF>
__device__ __forceinline__ void prefetch_dir(const HopArgs &A, int s, int nb, int rb) {
    if constexpr (PF != 0 && D < 8) {
        const long Vh = A.g.Vh;
        const char *ub = (const char *)A.gauge + ((size_t)D * 9 * Vh + s) * LIO<G>::ELEM;
#pragma unroll
        for (int k = 0; k < 9; ++k) prefetch_line<PF>(ub + (size_t)k * Vh * LIO<G>::ELEM);
        constexpr int NCH = SIO<SIn>::NCH;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int rhs = tile_rhs(A, rb, r, R);
            if (rhs >= 0) {
                const uint4 *q = (const uint4 *)A.in + (size_t)rhs * NCH * Vh + nb;
#pragma unroll
                for (int k = 0; k < NCH; ++k) prefetch_line<PF>(q + (size_t)k * Vh);
            }
        }
    }
}

template <typename SIn, typename G, int R, int D, bool DAG, int PF = 0>
__device__ __forceinline__ void hop_dir_f2(const HopArgs &A, int s, int nb, int rb, float2 acc[][12],
                                           int nb_next = 0) {
    prefetch_dir<SIn, G, R, D + 1, PF>(A, s, nb_next, rb);
    constexpr int MU = D & 3;
    constexpr bool FWD = D < 4;
    constexpr int SIGN = (FWD != DAG) ? -1 : +1;
    const long Vh = A.g.Vh;
    cx<float> u[9];
    LIO<G>::load((const char *)A.gauge + (size_t)D * 9 * Vh * LIO<G>::ELEM, Vh, s, u);
    float2 ur[9], ui[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { ur[k] = f2(u[k].re, u[k].re); ui[k] = f2(-u[k].im, u[k].im); }
    constexpr int NCH = SIO<SIn>::NCH;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = tile_rhs(A, rb, r, R);
        if (rhs >= 0) {
            float2 psi[12], h[6], hs[6], uh[6];
            load_f2<SIn>((const uint4 *)A.in + (size_t)rhs * NCH * Vh, Vh, nb, psi);
            proj_f2<MU, SIGN>(psi, h);
#pragma unroll
            for (int k = 0; k < 6; ++k) hs[k] = sw(h[k]);
#pragma unroll
            for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float2 a = __fmul2_rn(ur[3 * i], h[3 * sp]);
                    a = __ffma2_rn(ui[3 * i], hs[3 * sp], a);
#pragma unroll
                    for (int j = 1; j < 3; ++j) {
                        a = __ffma2_rn(ur[3 * i + j], h[3 * sp + j], a);
                        a = __ffma2_rn(ui[3 * i + j], hs[3 * sp + j], a);
                    }
                    uh[3 * sp + i] = a;
                }
            recon_f2<MU, SIGN>(acc[r], uh);
        }
    }
}

// Split form of one direction for the software-pipelined variant: the loads of
// direction d+1 (link + R neighbour spinors) are issued before the arithmetic
// of direction d, so each thread keeps two directions of loads in flight.
template <typename SIn, typename G, int R, int D>
__device__ __forceinline__ void load_dir_f2(const HopArgs &A, int s, int nb, int rb, cx<float> u[9],
                                            float2 psi[][12]) {
    const long Vh = A.g.Vh;
    LIO<G>::load((const char *)A.gauge + (size_t)D * 9 * Vh * LIO<G>::ELEM, Vh, s, u);
    constexpr int NCH = SIO<SIn>::NCH;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = tile_rhs(A, rb, r, R);
        if (rhs >= 0) load_f2<SIn>((const uint4 *)A.in + (size_t)rhs * NCH * Vh, Vh, nb, psi[r]);
    }
}

template <int R, int D, bool DAG>
__device__ __forceinline__ void compute_dir_f2(const HopArgs &A, int rb, const cx<float> u[9], float2 psi[][12],
                                               float2 acc[][12]) {
    constexpr int MU = D & 3;
    constexpr bool FWD = D < 4;
    constexpr int SIGN = (FWD != DAG) ? -1 : +1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (tile_rhs(A, rb, r, R) >= 0) {
            float2 h[6], hs[6], uh[6];
            proj_f2<MU, SIGN>(psi[r], h);
#pragma unroll
            for (int k = 0; k < 6; ++k) hs[k] = sw(h[k]);
#pragma unroll
            for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float2 a = __fmul2_rn(f2(u[3 * i].re, u[3 * i].re), h[3 * sp]);
                    a = __ffma2_rn(f2(-u[3 * i].im, u[3 * i].im), hs[3 * sp], a);
#pragma unroll
                    for (int j = 1; j < 3; ++j) {
                        a = __ffma2_rn(f2(u[3 * i + j].re, u[3 * i + j].re), h[3 * sp + j], a);
                        a = __ffma2_rn(f2(-u[3 * i + j].im, u[3 * i + j].im), hs[3 * sp + j], a);
                    }
                    uh[3 * sp + i] = a;
                }
            recon_f2<MU, SIGN>(acc[r], uh);
        }
    }
}

template <typename SIn, typename G, int R, bool DAG>
__device__ __forceinline__ void hop_dirs_pipelined(const HopArgs &A, int s, int rb, const int nb[8],
                                                   float2 acc[][12]) {
    cx<float> ua[9], ub[9];
    float2 pa[R][12], pb[R][12];
    load_dir_f2<SIn, G, R, 0>(A, s, nb[0], rb, ua, pa);
    load_dir_f2<SIn, G, R, 1>(A, s, nb[1], rb, ub, pb);
    compute_dir_f2<R, 0, DAG>(A, rb, ua, pa, acc);
    load_dir_f2<SIn, G, R, 2>(A, s, nb[2], rb, ua, pa);
    compute_dir_f2<R, 1, DAG>(A, rb, ub, pb, acc);
    load_dir_f2<SIn, G, R, 3>(A, s, nb[3], rb, ub, pb);
    compute_dir_f2<R, 2, DAG>(A, rb, ua, pa, acc);
    load_dir_f2<SIn, G, R, 4>(A, s, nb[4], rb, ua, pa);
    compute_dir_f2<R, 3, DAG>(A, rb, ub, pb, acc);
    load_dir_f2<SIn, G, R, 5>(A, s, nb[5], rb, ub, pb);
    compute_dir_f2<R, 4, DAG>(A, rb, ua, pa, acc);
    load_dir_f2<SIn, G, R, 6>(A, s, nb[6], rb, ua, pa);
    compute_dir_f2<R, 5, DAG>(A, rb, ub, pb, acc);
    load_dir_f2<SIn, G, R, 7>(A, s, nb[7], rb, ub, pb);
    compute_dir_f2<R, 6, DAG>(A, rb, ua, pa, acc);
    compute_dir_f2<R, 7, DAG>(A, rb, ub, pb, acc);
}

// one output site s for RHS tile rb
template <typename SIn, typename SOut, typename SW, typename G, int R, bool DAG, bool PIPE = false, int PF = 0>
__device__ __forceinline__ void hop_site_f2(const HopArgs &A, int rb, int s) {
    const Geom &g = A.g;
    int x, y, z, t;
    eo_coords(g, A.p, s, x, y, z, t);
    const int xp = x + 1 == g.X ? 0 : x + 1, xm = x == 0 ? g.X - 1 : x - 1;
    const int yp = y + 1 == g.Y ? 0 : y + 1, ym = y == 0 ? g.Y - 1 : y - 1;
    const int zp = z + 1 == g.Z ? 0 : z + 1, zm = z == 0 ? g.Z - 1 : z - 1;
    const int tp = t + 1 == g.T ? 0 : t + 1, tm = t == 0 ? g.T - 1 : t - 1;
    float2 acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = f2(0.f, 0.f);
    if constexpr (PIPE) {
        const int nb[8] = {eo_index(g, xp, y, z, t), eo_index(g, x, yp, z, t), eo_index(g, x, y, zp, t),
                           eo_index(g, x, y, z, tp), eo_index(g, xm, y, z, t), eo_index(g, x, ym, z, t),
                           eo_index(g, x, y, zm, t), eo_index(g, x, y, z, tm)};
        hop_dirs_pipelined<SIn, G, R, DAG>(A, s, rb, nb, acc);
    } else if constexpr (PF != 0) {
        const int nb[8] = {eo_index(g, xp, y, z, t), eo_index(g, x, yp, z, t), eo_index(g, x, y, zp, t),
                           eo_index(g, x, y, z, tp), eo_index(g, xm, y, z, t), eo_index(g, x, ym, z, t),
                           eo_index(g, x, y, zm, t), eo_index(g, x, y, z, tm)};
        prefetch_dir<SIn, G, R, 0, PF>(A, s, nb[0], rb);
        hop_dir_f2<SIn, G, R, 0, DAG, PF>(A, s, nb[0], rb, acc, nb[1]);
        hop_dir_f2<SIn, G, R, 1, DAG, PF>(A, s, nb[1], rb, acc, nb[2]);
        hop_dir_f2<SIn, G, R, 2, DAG, PF>(A, s, nb[2], rb, acc, nb[3]);
        hop_dir_f2<SIn, G, R, 3, DAG, PF>(A, s, nb[3], rb, acc, nb[4]);
        hop_dir_f2<SIn, G, R, 4, DAG, PF>(A, s, nb[4], rb, acc, nb[5]);
        hop_dir_f2<SIn, G, R, 5, DAG, PF>(A, s, nb[5], rb, acc, nb[6]);
        hop_dir_f2<SIn, G, R, 6, DAG, PF>(A, s, nb[6], rb, acc, nb[7]);
        hop_dir_f2<SIn, G, R, 7, DAG, PF>(A, s, nb[7], rb, acc);
    } else {
        hop_dir_f2<SIn, G, R, 0, DAG>(A, s, eo_index(g, xp, y, z, t), rb, acc);
        hop_dir_f2<SIn, G, R, 1, DAG>(A, s, eo_index(g, x, yp, z, t), rb, acc);
        hop_dir_f2<SIn, G, R, 2, DAG>(A, s, eo_index(g, x, y, zp, t), rb, acc);
        hop_dir_f2<SIn, G, R, 3, DAG>(A, s, eo_index(g, x, y, z, tp), rb, acc);
        hop_dir_f2<SIn, G, R, 4, DAG>(A, s, eo_index(g, xm, y, z, t), rb, acc);
        hop_dir_f2<SIn, G, R, 5, DAG>(A, s, eo_index(g, x, ym, z, t), rb, acc);
        hop_dir_f2<SIn, G, R, 6, DAG>(A, s, eo_index(g, x, y, zm, t), rb, acc);
        hop_dir_f2<SIn, G, R, 7, DAG>(A, s, eo_index(g, x, y, z, tm), rb, acc);
    }
    const long Vh = g.Vh;
    constexpr int NO = SIO<SOut>::NCH, NW = SIO<SW>::NCH;
    const float2 a2 = f2((float)A.a, (float)A.a), b2 = f2((float)A.b, (float)A.b), c2 = f2((float)A.c, (float)A.c);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = tile_rhs(A, rb, r, R);
        if (rhs < 0) break;
        float2 o[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = __fmul2_rn(b2, acc[r][k]);
        if (A.w) {
            float2 wv[12];
            load_f2<SW>((const uint4 *)A.w + (size_t)rhs * NW * Vh, Vh, s, wv);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = __ffma2_rn(a2, wv[k], o[k]);
        }
        if (A.w2) {
            float2 wv[12];
            load_f2<SW>((const uint4 *)A.w2 + (size_t)rhs * NW * Vh, Vh, s, wv);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = __ffma2_rn(c2, wv[k], o[k]);
        }
        cx<float> oc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) oc[k] = cmake(o[k].x, o[k].y);
        SIO<SOut>::store((uint4 *)A.out + (size_t)rhs * NO * Vh, Vh, s, oc);
    }
}

template <typename SIn, typename SOut, typename SW, typename G, int R, bool DAG, bool PIPE, int PF = 0>
__global__ void __launch_bounds__(256) hop_kernel_f2(HopArgs A) {
    pdl_wait();
    const int nsb = gridDim.x / A.nrb;
    const int rb = A.rhs_major ? blockIdx.x / nsb : blockIdx.x % A.nrb;
    const int s = (A.rhs_major ? blockIdx.x % nsb : blockIdx.x / A.nrb) * blockDim.x + threadIdx.x;
    if (s < A.g.Vh && tile_rhs(A, rb, 0, R) >= 0) hop_site_f2<SIn, SOut, SW, G, R, DAG, PIPE, PF>(A, rb, s);
}

// Register-capped variant: the same site body with __launch_bounds__(128,
// MINB), so that MINB CTAs of 128 threads fit per SM (more resident warps to
// hide the neighbour-load latency, at the price of spills if the cap is
// below what the body needs); site tile fastest in the block order
// A.rhs_major = 1: all site tiles of one RHS tile, then the next RHS tile;
// A.rhs_major = GR >= 2: RHS tiles in groups of GR, and within a group the GR
// tiles of one site tile together, then the next site tile.  Grouping bounds
// the links' DRAM traffic (re-read once per group instead of once per RHS
// tile when the links exceed L2) while the inputs the group's resident blocks
// need from the neighbouring timeslices still fit in L2.
template <typename SIn, typename SOut, typename SW, typename G, int R, bool DAG, int MINB>
__global__ void __launch_bounds__(128, MINB) hop_kernel_f2_cap(HopArgs A) {
    const int nsb = (A.g.Vh + blockDim.x - 1) / blockDim.x;
    int rb, sb;
    if (A.rhs_major >= 2) {
        const int GR = A.rhs_major, per = GR * nsb;
        const int grp = blockIdx.x / per, rem = blockIdx.x - grp * per;
        sb = rem / GR;
        rb = grp * GR + (rem - sb * GR);
        if (rb >= A.nrb) return;
    } else {
        rb = blockIdx.x / nsb;
        sb = blockIdx.x - rb * nsb;
    }
    const int s = sb * blockDim.x + threadIdx.x;
    if (s < A.g.Vh && tile_rhs(A, rb, 0, R) >= 0) hop_site_f2<SIn, SOut, SW, G, R, DAG, false, 0>(A, rb, s);
}

// Persistent batched stencil over several lattices: one launch walks
// a static work list of (lattice, site tile, RHS tile) items -- the items of
// lattice j are the blocks [base_j, base_j + blocks_j) -- with a grid sized to
// the resident CTAs of the GPU; CTA i takes items i, i + gridDim.x, ...  No
// atomics and no waits: the assignment is fixed, so the result is
// deterministic and nothing can hang.
template <typename SIn, typename SOut, typename SW, typename G, int R>
__global__ void __launch_bounds__(128) hop_batched_f2(const __grid_constant__ HopBatch B) {
    for (int item = blockIdx.x; item < B.total; item += gridDim.x) {
        int j = 0, base = 0;
        while (j + 1 < B.njobs && item - base >= B.blocks[j]) { base += B.blocks[j]; ++j; }
        const HopArgs &A = B.job[j];
        const int lb = item - base;
        const int rb = lb % A.nrb;
        const int s = (lb / A.nrb) * blockDim.x + threadIdx.x;
        if (s < A.g.Vh) hop_site_f2<SIn, SOut, SW, G, R, false>(A, rb, s);
    }
}

template <typename SIn, typename SOut, typename SW, typename G>
cudaError_t launch_hop_batched(HopBatch B, int R, cudaStream_t st) {
    if (R != 1 && R != 2 && R != 4) R = 2;
    const int th = 128;
    B.total = 0;
    for (int j = 0; j < B.njobs; ++j) {
        B.job[j].nrb = (B.job[j].nrhs + R - 1) / R;
        B.blocks[j] = ((B.job[j].g.Vh + th - 1) / th) * B.job[j].nrb;
        B.total += B.blocks[j];
    }
    if (B.total == 0) return cudaSuccess;
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
#define WD_HB_CASE(RR)                                                                             \
    if (R == RR) {                                                                                 \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hop_batched_f2<SIn, SOut, SW, G, RR>, th, 0); \
        int grid = sms * (per > 0 ? per : 1);                                                      \
        if (grid > B.total) grid = B.total;                                                        \
        hop_batched_f2<SIn, SOut, SW, G, RR><<<grid, th, 0, st>>>(B);                              \
    }
    WD_HB_CASE(1) WD_HB_CASE(2) WD_HB_CASE(4)
#undef WD_HB_CASE
    return cudaGetLastError();
}

template cudaError_t launch_hop_batched<float, float, float, float>(HopBatch, int, cudaStream_t);
template cudaError_t launch_hop_batched<bf16, bf16, bf16, bf16>(HopBatch, int, cudaStream_t);
template cudaError_t launch_hop_batched<bf16, float, bf16, bf16>(HopBatch, int, cudaStream_t);

// ---- staged variant: timeslices through shared memory by bulk async copies ----
// For many right-hand sides on lattices with small timeslices.  A CTA walks a
// column of consecutive timeslices t in [ta, tb) for one group of R RHS; a ring
// of 4 shared-memory slots holds the input (other parity) timeslices t-1, t,
// t+1 and the prefetched t+2, each brought in by cp.async.bulk (TMA, 1D) on an
// mbarrier.  All 8 neighbour spinors come from shared memory; every input
// spinor of the column is read from global memory once; the loads in flight
// cost no registers.  Links and the epilogue addends are read from global.
static constexpr int ST_SLOTS = 4;
static constexpr long ST_SPIN = 1L << 24;

__device__ __forceinline__ uint32_t st_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool st_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = st_u32(bar);
    for (long i = 0; i < ST_SPIN; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

// Bulk copies of input timeslice u (unwrapped; slot (u - ta + 1) & 3) for the nr
// RHS of the group: NCH rows of Sl 16-byte chunks per RHS.  Thread 0 only.
template <int NCH>
__device__ __forceinline__ void st_issue(unsigned char *smem, size_t slot_bytes, uint64_t *full, int *loads,
                                         const uint4 *in, long Vh, int Sl, int T, int ta, int u, int r0, int nr) {
    const int q = (u - ta + 1) & 3;
    const int tt = ((u % T) + T) % T;
    const uint32_t bytes = (uint32_t)nr * NCH * Sl * 16;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(st_u32(&full[q])), "r"(bytes) : "memory");
    for (int r = 0; r < nr; ++r)
        for (int k = 0; k < NCH; ++k) {
            unsigned char *dst = smem + q * slot_bytes + (size_t)(r * NCH + k) * Sl * 16;
            const uint4 *src = in + ((size_t)(r0 + r) * NCH + k) * Vh + (size_t)tt * Sl;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(st_u32(dst)), "l"((uint64_t)src), "r"((uint32_t)Sl * 16), "r"(st_u32(&full[q]))
                         : "memory");
        }
    loads[q] += 1;
}

// one site's 12 complex components from a shared-memory slice [k][Sl] of 16-byte chunks
template <typename S> __device__ __forceinline__ void load_smem_f2(const unsigned char *p, int Sl, int o, float2 v[12]);
template <> __device__ __forceinline__ void load_smem_f2<float>(const unsigned char *p, int Sl, int o, float2 v[12]) {
    const float4 *q = (const float4 *)p + o;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 a = q[k * Sl];
        v[2 * k] = f2(a.x, a.y);
        v[2 * k + 1] = f2(a.z, a.w);
    }
}
template <> __device__ __forceinline__ void load_smem_f2<bf16>(const unsigned char *p, int Sl, int o, float2 v[12]) {
    const uint4 *q = (const uint4 *)p + o;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 a = q[k * Sl];
        const __nv_bfloat162 *h = (const __nv_bfloat162 *)&a;
#pragma unroll
        for (int j = 0; j < 4; ++j) v[4 * k + j] = __bfloat1622float2(h[j]);
    }
}

template <typename SIn, typename SOut, typename SW, typename G, int R, bool DAG>
__global__ void __launch_bounds__(256, 1) hop_staged_f2(HopArgs A, int tlen) {
    constexpr int NCH = SIO<SIn>::NCH;
    const Geom &g = A.g;
    const long Vh = g.Vh;
    const int T = g.T, Sl = g.Vh / g.T;
    const int rg = blockIdx.x % A.nrb, tcol = blockIdx.x / A.nrb;
    const int ta = tcol * tlen, tb = min(ta + tlen, T);
    const int r0 = rg * R, nr = min(R, A.nrhs - r0);
    const size_t slot_bytes = (size_t)R * NCH * Sl * 16;
    extern __shared__ __align__(128) unsigned char st_smem[];
    uint64_t *full = (uint64_t *)(st_smem + ST_SLOTS * slot_bytes);
    __shared__ int s_fail;
    __shared__ int s_loads[ST_SLOTS];
    if (threadIdx.x == 0) {
        for (int q = 0; q < ST_SLOTS; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(st_u32(&full[q])));
            s_loads[q] = 0;
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int u = ta - 1; u <= min(ta + 2, tb); ++u)
            st_issue<NCH>(st_smem, slot_bytes, full, s_loads, (const uint4 *)A.in, Vh, Sl, T, ta, u, r0, nr);
    for (int t = ta; t < tb; ++t) {
        // slices t-1, t, t+1 must have landed
        bool ok = true;
        for (int u = t - 1; u <= t + 1; ++u)
            ok = ok && st_wait(&full[(u - ta + 1) & 3], ((u - ta + 1) >> 2) & 1);
        if (!ok) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const unsigned char *sm = st_smem + ((t - 1 - ta + 1) & 3) * slot_bytes;
        const unsigned char *s0 = st_smem + ((t - ta + 1) & 3) * slot_bytes;
        const unsigned char *sp = st_smem + ((t + 1 - ta + 1) & 3) * slot_bytes;
        for (int so = threadIdx.x; so < Sl; so += blockDim.x) {
            const int s = t * Sl + so;
            int x, y, z, tt;
            eo_coords(g, A.p, s, x, y, z, tt);
            const int xp = x + 1 == g.X ? 0 : x + 1, xm = x == 0 ? g.X - 1 : x - 1;
            const int yp = y + 1 == g.Y ? 0 : y + 1, ym = y == 0 ? g.Y - 1 : y - 1;
            const int zp = z + 1 == g.Z ? 0 : z + 1, zm = z == 0 ? g.Z - 1 : z - 1;
            const int base = t * Sl;
            const int onb[8] = {eo_index(g, xp, y, z, t) - base, eo_index(g, x, yp, z, t) - base,
                                eo_index(g, x, y, zp, t) - base, eo_index(g, x, y, z, 0),
                                eo_index(g, xm, y, z, t) - base, eo_index(g, x, ym, z, t) - base,
                                eo_index(g, x, y, zm, t) - base, eo_index(g, x, y, z, 0)};
            float2 acc[R][12];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int k = 0; k < 12; ++k) acc[r][k] = f2(0.f, 0.f);
#define WD_ST_DIR(D, SLOT)                                                                         \
            {                                                                                      \
                cx<float> u[9];                                                                    \
                LIO<G>::load((const char *)A.gauge + (size_t)(D) * 9 * Vh * LIO<G>::ELEM, Vh, s, u); \
                float2 psi[R][12];                                                                 \
                _Pragma("unroll") for (int r = 0; r < R; ++r)                                      \
                    if (r < nr) load_smem_f2<SIn>((SLOT) + (size_t)r * NCH * Sl * 16, Sl, onb[D], psi[r]); \
                compute_dir_f2<R, D, DAG>(A, rg, u, psi, acc);                                     \
                asm volatile("" ::: "memory");                                                     \
            }
            WD_ST_DIR(0, s0) WD_ST_DIR(1, s0) WD_ST_DIR(2, s0) WD_ST_DIR(3, sp)
            WD_ST_DIR(4, s0) WD_ST_DIR(5, s0) WD_ST_DIR(6, s0) WD_ST_DIR(7, sm)
#undef WD_ST_DIR
            constexpr int NO = SIO<SOut>::NCH, NW = SIO<SW>::NCH;
            const float2 a2 = f2((float)A.a, (float)A.a), b2 = f2((float)A.b, (float)A.b), c2 = f2((float)A.c, (float)A.c);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r >= nr) break;
                const int rhs = r0 + r;
                float2 o[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) o[k] = __fmul2_rn(b2, acc[r][k]);
                if (A.w) {
                    float2 wv[12];
                    load_f2<SW>((const uint4 *)A.w + (size_t)rhs * NW * Vh, Vh, s, wv);
#pragma unroll
                    for (int k = 0; k < 12; ++k) o[k] = __ffma2_rn(a2, wv[k], o[k]);
                }
                if (A.w2) {
                    float2 wv[12];
                    load_f2<SW>((const uint4 *)A.w2 + (size_t)rhs * NW * Vh, Vh, s, wv);
#pragma unroll
                    for (int k = 0; k < 12; ++k) o[k] = __ffma2_rn(c2, wv[k], o[k]);
                }
                cx<float> oc[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) oc[k] = cmake(o[k].x, o[k].y);
                SIO<SOut>::store((uint4 *)A.out + (size_t)rhs * NO * Vh, Vh, s, oc);
            }
        }
        // every thread is done with slot(t-1): order its reads before the async refill
        __syncthreads();
        if (threadIdx.x == 0 && t + 3 <= tb) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            st_issue<NCH>(st_smem, slot_bytes, full, s_loads, (const uint4 *)A.in, Vh, Sl, T, ta, t + 3, r0, nr);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) {
        if (A.err) atomicExch(A.err, 1);
        // copies already issued must land before the shared memory is released
        for (int q = 0; q < ST_SLOTS; ++q)
            if (s_loads[q] > 0) st_wait(&full[q], (s_loads[q] - 1) & 1);
    }
}

// ---- plane-walk variant: persistent CTAs walk z through a timeslice --------
// A unit is (RHS tile of 2, timeslice t); a CTA takes units u = blockIdx.x,
// blockIdx.x + gridDim.x, ... and walks z = 0 .. Z-1 through each.  A ring of
// 4 shared-memory slots holds the tile's input (other parity) x-y planes
// z-1, z, z+1 and the next plane in flight, each a set of 1D cp.async.bulk
// copies (one per RHS and 16-byte channel; a plane is contiguous in every
// channel) completing on the slot's mbarrier; all waits are bounded.  The
// x, y and z neighbours of a site come from shared memory, so every input
// spinor crosses L2 once for them; the t neighbours, the links and the
// addends are plain loads.  One thread per (plane site, RHS of the tile).
// Units go in bands of W timeslices with all RHS tiles of a band together:
// the tiles running at one time share the band's links in L2, and the t
// neighbours of a unit are planes that the units at t - 1 and t + 1 stage
// at about the same time.
static constexpr int PW_SLOTS = 4;

__device__ __forceinline__ void pw_unit(const HopArgs &A, int W, int ntiles, int u, int &rb, int &t) {
    const int per = ntiles * W, band = u / per, rem = u - band * per;
    rb = rem / W;
    t = band * W + (rem - rb * W);
}

// plane j (-1 .. Z) of unit u into slot n & 3 (thread 0 only)
__device__ __forceinline__ void pw_issue(const HopArgs &A, unsigned char *smem, size_t slot_bytes, uint64_t *full,
                                        int *loads, int S, int W, int ntiles, int u, int j, int n) {
    int rb, t;
    pw_unit(A, W, ntiles, u, rb, t);
    const int Z = A.g.Z, z = (j + Z) % Z, q = n & (PW_SLOTS - 1);
    const long Vh = A.g.Vh;
    const size_t off = ((size_t)t * Z + z) * S;
    int nr = 0;
    for (int r = 0; r < 2; ++r) nr += tile_rhs(A, rb, r, 2) >= 0;
    const uint32_t bytes = (uint32_t)nr * 6 * S * 16;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(st_u32(&full[q])), "r"(bytes) : "memory");
    for (int r = 0; r < 2; ++r) {
        const int rhs = tile_rhs(A, rb, r, 2);
        if (rhs < 0) continue;
        for (int k = 0; k < 6; ++k) {
            unsigned char *dst = smem + q * slot_bytes + (size_t)(r * 6 + k) * S * 16;
            const uint4 *src = (const uint4 *)A.in + ((size_t)rhs * 6 + k) * Vh + off;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(st_u32(dst)), "l"((uint64_t)src), "r"((uint32_t)S * 16), "r"(st_u32(&full[q]))
                         : "memory");
        }
    }
    loads[q] += 1;
}

// one hop term: acc += (1 -/+ g_mu) U psi for the link u (split as the f32x2
// multiplier pairs ur, ui) and the neighbour spinor psi
template <int MU, int SIGN>
__device__ __forceinline__ void pw_term(const float2 ur[9], const float2 ui[9], const float2 psi[12],
                                        float2 acc[12]) {
    float2 h[6], hs[6], uh[6];
    proj_f2<MU, SIGN>(psi, h);
#pragma unroll
    for (int k = 0; k < 6; ++k) hs[k] = sw(h[k]);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float2 a = __fmul2_rn(ur[3 * i], h[3 * sp]);
            a = __ffma2_rn(ui[3 * i], hs[3 * sp], a);
#pragma unroll
            for (int j = 1; j < 3; ++j) {
                a = __ffma2_rn(ur[3 * i + j], h[3 * sp + j], a);
                a = __ffma2_rn(ui[3 * i + j], hs[3 * sp + j], a);
            }
            uh[3 * sp + i] = a;
        }
    recon_f2<MU, SIGN>(acc, uh);
}

template <int D, bool DAG>
__device__ __forceinline__ void pw_dir(const HopArgs &A, long s, const float2 psi[12], float2 acc[12]) {
    constexpr int MU = D & 3;
    constexpr int SIGN = ((D < 4) != DAG) ? -1 : +1;
    const long Vh = A.g.Vh;
    cx<float> u[9];
    LIO<float>::load((const char *)A.gauge + (size_t)D * 9 * Vh * LIO<float>::ELEM, Vh, s, u);
    float2 ur[9], ui[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { ur[k] = f2(u[k].re, u[k].re); ui[k] = f2(-u[k].im, u[k].im); }
    pw_term<MU, SIGN>(ur, ui, psi, acc);
}

template <bool DAG>
__global__ void __launch_bounds__(576, 1) hop_plane_f2(HopArgs A, int W) {
    const Geom &g = A.g;
    const long Vh = g.Vh;
    const int Z = g.Z, T = g.T, S = (int)(Vh / ((long)Z * T));
    const size_t slot_bytes = (size_t)2 * 6 * S * 16;
    extern __shared__ __align__(128) unsigned char pw_smem[];
    uint64_t *full = (uint64_t *)(pw_smem + PW_SLOTS * slot_bytes);
    __shared__ int s_fail;
    __shared__ int s_loads[PW_SLOTS];
    const int nact = A.alist ? __ldg(A.acount) : A.nrhs;
    const int ntiles = (nact + 1) / 2, nunits = ntiles * T;
    if ((int)blockIdx.x >= nunits) return;                 // uniform in the CTA, before any barrier
    const int my_units = (nunits - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
    const int nitems = my_units * (Z + 2);
    const int tid = threadIdx.x, rs = tid / S, so = tid - rs * S;
    int issued = 0;                                        // thread 0's count of plane copies issued
    if (tid == 0) {
        for (int q = 0; q < PW_SLOTS; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(st_u32(&full[q])));
            s_loads[q] = 0;
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (; issued < nitems && issued < PW_SLOTS; ++issued)
            pw_issue(A, pw_smem, slot_bytes, full, s_loads, S, W, ntiles, blockIdx.x + (issued / (Z + 2)) * gridDim.x,
                     issued % (Z + 2) - 1, issued);
    const float2 a2 = f2((float)A.a, (float)A.a), b2 = f2((float)A.b, (float)A.b), c2 = f2((float)A.c, (float)A.c);
    for (int k = 0; k < my_units && !s_fail; ++k) {
        int rb, t;
        pw_unit(A, W, ntiles, blockIdx.x + k * gridDim.x, rb, t);
        const int rhs = rs < 2 ? tile_rhs(A, rb, rs, 2) : -1;
        const int tp = t + 1 == T ? 0 : t + 1, tm = t == 0 ? T - 1 : t - 1;
        for (int z = 0; z < Z; ++z) {
            const int n0 = k * (Z + 2) + z;                // item of plane z - 1
            bool ok = true;
            for (int m = 0; m < 3; ++m) ok = ok && st_wait(&full[(n0 + m) & (PW_SLOTS - 1)], ((n0 + m) >> 2) & 1);
            if (!ok) s_fail = 1;
            __syncthreads();
            if (s_fail) break;
            if (rhs >= 0) {
                const unsigned char *pm = pw_smem + ((n0) & (PW_SLOTS - 1)) * slot_bytes + (size_t)rs * 6 * S * 16;
                const unsigned char *p0 = pw_smem + ((n0 + 1) & (PW_SLOTS - 1)) * slot_bytes + (size_t)rs * 6 * S * 16;
                const unsigned char *pp = pw_smem + ((n0 + 2) & (PW_SLOTS - 1)) * slot_bytes + (size_t)rs * 6 * S * 16;
                const int xh = so % g.Xh, y = so / g.Xh;
                const int x = 2 * xh + ((A.p + y + z + t) & 1);
                const int xp = x + 1 == g.X ? 0 : x + 1, xm = x == 0 ? g.X - 1 : x - 1;
                const int yp = y + 1 == g.Y ? 0 : y + 1, ym = y == 0 ? g.Y - 1 : y - 1;
                const long s = ((long)t * Z + z) * S + so;
                const uint4 *in = (const uint4 *)A.in + (size_t)rhs * 6 * Vh;
                float2 acc[12];
#pragma unroll
                for (int q = 0; q < 12; ++q) acc[q] = f2(0.f, 0.f);
                float2 psi[12];
                load_f2<float>(in, Vh, ((long)tp * Z + z) * S + so, psi);
                pw_dir<3, DAG>(A, s, psi, acc);
                load_f2<float>(in, Vh, ((long)tm * Z + z) * S + so, psi);
                pw_dir<7, DAG>(A, s, psi, acc);
                load_smem_f2<float>(p0, S, y * g.Xh + (xp >> 1), psi);
                pw_dir<0, DAG>(A, s, psi, acc);
                load_smem_f2<float>(p0, S, y * g.Xh + (xm >> 1), psi);
                pw_dir<4, DAG>(A, s, psi, acc);
                load_smem_f2<float>(p0, S, yp * g.Xh + xh, psi);
                pw_dir<1, DAG>(A, s, psi, acc);
                load_smem_f2<float>(p0, S, ym * g.Xh + xh, psi);
                pw_dir<5, DAG>(A, s, psi, acc);
                load_smem_f2<float>(pp, S, so, psi);
                pw_dir<2, DAG>(A, s, psi, acc);
                load_smem_f2<float>(pm, S, so, psi);
                pw_dir<6, DAG>(A, s, psi, acc);
                float2 o[12];
#pragma unroll
                for (int q = 0; q < 12; ++q) o[q] = __fmul2_rn(b2, acc[q]);
                if (A.w) {
                    float2 wv[12];
                    load_f2<float>((const uint4 *)A.w + (size_t)rhs * 6 * Vh, Vh, s, wv);
#pragma unroll
                    for (int q = 0; q < 12; ++q) o[q] = __ffma2_rn(a2, wv[q], o[q]);
                }
                if (A.w2) {
                    float2 wv[12];
                    load_f2<float>((const uint4 *)A.w2 + (size_t)rhs * 6 * Vh, Vh, s, wv);
#pragma unroll
                    for (int q = 0; q < 12; ++q) o[q] = __ffma2_rn(c2, wv[q], o[q]);
                }
                cx<float> oc[12];
#pragma unroll
                for (int q = 0; q < 12; ++q) oc[q] = cmake(o[q].x, o[q].y);
                SIO<float>::store((uint4 *)A.out + (size_t)rhs * 6 * Vh, Vh, s, oc);
            }
            // every thread is done with plane z - 1: order its reads before the
            // async refill, then top the ring up from the first item still needed
            __syncthreads();
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const int need = z + 1 < Z ? n0 + 1 : n0 + 3;
                for (; issued < nitems && issued < need + PW_SLOTS; ++issued)
                    pw_issue(A, pw_smem, slot_bytes, full, s_loads, S, W, ntiles,
                             blockIdx.x + (issued / (Z + 2)) * gridDim.x, issued % (Z + 2) - 1, issued);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && s_fail) {
        if (A.err) atomicExch(A.err, 1);
        // copies already issued must land before the shared memory is released
        for (int q = 0; q < PW_SLOTS; ++q)
            if (s_loads[q] > 0) st_wait(&full[q], (s_loads[q] - 1) & 1);
    }
}

size_t hop_plane_smem(const Geom &g) {
    return (size_t)PW_SLOTS * 2 * 6 * (g.Vh / ((long)g.Z * g.T)) * 16 + PW_SLOTS * 8;
}

template <typename SIn, typename SOut, typename SW, typename G>
cudaError_t launch_hop_plane(const HopArgs &A0, bool dag, cudaStream_t st) {
    if constexpr (!(std::is_same<SIn, float>::value && std::is_same<SOut, float>::value &&
                    std::is_same<SW, float>::value && std::is_same<G, float>::value)) {
        return cudaErrorNotSupported;
    } else {
        HopArgs A = A0;
        if (A.nrhs <= 0) return cudaSuccess;
        const int S = (int)(A.g.Vh / ((long)A.g.Z * A.g.T));
        const size_t smem = hop_plane_smem(A.g);
        const int th = 2 * S;
        if (th > 576 || A.g.Z < 3 || smem > 227 * 1024) return cudaErrorNotSupported;
        int W = 1;                                           // the largest divisor of T up to 12
        for (int w = 1; w <= 12 && w <= A.g.T; ++w)
            if (A.g.T % w == 0) W = w;
        int dev = 0, sms = 148, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int ntiles = (A.nrhs + 1) / 2;
        auto kern = dag ? hop_plane_f2<true> : hop_plane_f2<false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, th, smem);
        if (per < 1) return cudaErrorNotSupported;
        long grid = (long)sms * per;
        if (grid > (long)ntiles * A.g.T) grid = (long)ntiles * A.g.T;
        kern<<<(unsigned)grid, th, smem, st>>>(A, W);
        return cudaGetLastError();
    }
}

size_t hop_staged_smem(const HopArgs &A, int R, int nch) {
    if (A.g.Vh % A.g.T) return 0;
    return (size_t)ST_SLOTS * R * nch * (A.g.Vh / A.g.T) * 16 + ST_SLOTS * 8;
}

template <typename SIn, typename SOut, typename SW, typename G>
cudaError_t launch_hop_staged(const HopArgs &A0, int R, bool dag, cudaStream_t st) {
    if constexpr (std::is_same<typename RealOf<SIn>::type, double>::value) {
        return cudaErrorNotSupported;
    } else {
        HopArgs A = A0;
        if (A.nrhs <= 0) return cudaSuccess;
        if (R != 1 && R != 2 && R != 4) return cudaErrorNotSupported;
        const size_t smem = hop_staged_smem(A, R, SIO<SIn>::NCH);
        if (smem == 0 || smem > 200 * 1024 || A.g.T < 2) return cudaErrorNotSupported;
        A.nrb = (A.nrhs + R - 1) / R;
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = smem <= 100 * 1024 ? 2 : 1;
        const int target = sms * per_sm * 2;
        int ncolt = (target + A.nrb - 1) / A.nrb;
        if (ncolt > A.g.T) ncolt = A.g.T;
        if (ncolt < 1) ncolt = 1;
        const int tlen = (A.g.T + ncolt - 1) / ncolt;
        ncolt = (A.g.T + tlen - 1) / tlen;
        const unsigned grid = (unsigned)(A.nrb * ncolt);
        const int Sl = A.g.Vh / A.g.T;
        const int th = Sl >= 256 ? 256 : ((Sl + 31) / 32) * 32;
#define WD_ST_CASE(RR)                                                                                   \
        if (R == RR) {                                                                                   \
            if (dag) {                                                                                   \
                cudaFuncSetAttribute(hop_staged_f2<SIn, SOut, SW, G, RR, true>,                          \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
                hop_staged_f2<SIn, SOut, SW, G, RR, true><<<grid, th, smem, st>>>(A, tlen);              \
            } else {                                                                                     \
                cudaFuncSetAttribute(hop_staged_f2<SIn, SOut, SW, G, RR, false>,                         \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
                hop_staged_f2<SIn, SOut, SW, G, RR, false><<<grid, th, smem, st>>>(A, tlen);             \
            }                                                                                            \
        }
        WD_ST_CASE(1) WD_ST_CASE(2) WD_ST_CASE(4)
#undef WD_ST_CASE
        return cudaGetLastError();
    }
}

template <typename SIn, typename SOut, typename SW, typename G>
cudaError_t launch_hop(const HopArgs &A0, int R, bool dag, int threads, cudaStream_t st) {
    HopArgs A = A0;
    if (A.nrhs <= 0) return cudaSuccess;
    // R = 1, 2, 4: plain; R = 11, 12, 14: software-pipelined; R = 21, 22, 24:
    // timeslices staged through shared memory (FP32 arithmetic only); R = 31,
    // 32, 34 / 41, 42, 44: next-direction prefetch into L1 / L2; R = 51, 52,
    // 54: plain with the site tile fastest in the block order; R = 62: two RHS,
    // registers capped for 20 resident warps per SM; R = 63, 64, 65: the same
    // with the RHS tiles in groups of 4, 8, 16 (site tile fastest within a group);
    // R = 71: persistent plane walk with x-y planes staged in shared memory
    constexpr bool PACKED = !std::is_same<typename RealOf<SIn>::type, double>::value;
    if (R > 20 && R < 30) return launch_hop_staged<SIn, SOut, SW, G>(A, R - 20, dag, st);
    if (R == 71) return launch_hop_plane<SIn, SOut, SW, G>(A, dag, st);
    if (R >= 62 && R <= 65) {   // two RHS, register cap for 5 CTAs of 128 threads per SM
        // 62: site tile fastest; 63, 64, 65: RHS tiles in groups of 4, 8, 16
        if (!PACKED || threads > 128) return cudaErrorNotSupported;
        A.nrb = (A.nrhs + 1) / 2;
        const int nsb = (A.g.Vh + threads - 1) / threads;
        A.rhs_major = R == 62 ? 1 : 1 << (R - 61);
        const int GR = A.rhs_major, ngrp = (A.nrb + GR - 1) / GR;
        const dim3 grid((unsigned)(R == 62 ? (long)nsb * A.nrb : (long)ngrp * GR * nsb));
        if constexpr (PACKED) {
            if (dag) hop_kernel_f2_cap<SIn, SOut, SW, G, 2, true, 5><<<grid, threads, 0, st>>>(A);
            else hop_kernel_f2_cap<SIn, SOut, SW, G, 2, false, 5><<<grid, threads, 0, st>>>(A);
        }
        return cudaGetLastError();
    }
    if (R > 50) {   // R = 51, 52, 54: plain, site tile fastest
        if (!PACKED) return cudaErrorNotSupported;
        A.rhs_major = 1;
        R -= 50;
    }
    int pf = 0;
    if (R > 30) {
        if (!PACKED) return cudaErrorNotSupported;
        pf = R > 40 ? 2 : 1;
        R -= pf == 2 ? 40 : 30;
    }
    const bool pipe = R > 10;
    if (pipe) R -= 10;
    if (R != 1 && R != 2 && R != 4) R = 1;
    A.nrb = (A.nrhs + R - 1) / R;
    const int sblocks = (A.g.Vh + threads - 1) / threads;
    dim3 grid((unsigned)(sblocks * A.nrb));
#define WD_HOP_CASE(RR)                                                                                \
    if (R == RR) {                                                                                     \
        if constexpr (PACKED) {                                                                        \
            if (pf == 1) {                                                                             \
                if (dag) hop_kernel_f2<SIn, SOut, SW, G, RR, true, false, 1><<<grid, threads, 0, st>>>(A); \
                else hop_kernel_f2<SIn, SOut, SW, G, RR, false, false, 1><<<grid, threads, 0, st>>>(A); \
            } else if (pf == 2) {                                                                      \
                if (dag) hop_kernel_f2<SIn, SOut, SW, G, RR, true, false, 2><<<grid, threads, 0, st>>>(A); \
                else hop_kernel_f2<SIn, SOut, SW, G, RR, false, false, 2><<<grid, threads, 0, st>>>(A); \
            } else if (pipe) {                                                                         \
                if (dag) hop_kernel_f2<SIn, SOut, SW, G, RR, true, true><<<grid, threads, 0, st>>>(A); \
                else hop_kernel_f2<SIn, SOut, SW, G, RR, false, true><<<grid, threads, 0, st>>>(A);    \
            } else {                                                                                   \
                return dag ? launch_pdl(hop_kernel_f2<SIn, SOut, SW, G, RR, true, false>, grid, dim3(threads), \
                                        0, st, A)                                                      \
                           : launch_pdl(hop_kernel_f2<SIn, SOut, SW, G, RR, false, false>, grid,        \
                                        dim3(threads), 0, st, A);                                      \
            }                                                                                          \
        } else {                                                                                       \
            if (dag) hop_kernel<SIn, SOut, SW, G, RR, true><<<grid, threads, 0, st>>>(A);              \
            else hop_kernel<SIn, SOut, SW, G, RR, false><<<grid, threads, 0, st>>>(A);                 \
        }                                                                                              \
    }
    WD_HOP_CASE(1) WD_HOP_CASE(2) WD_HOP_CASE(4)
#undef WD_HOP_CASE
    return cudaGetLastError();
}

template cudaError_t launch_hop<double, double, double, double>(const HopArgs &, int, bool, int, cudaStream_t);
template cudaError_t launch_hop<float, float, float, float>(const HopArgs &, int, bool, int, cudaStream_t);
template cudaError_t launch_hop<bf16, bf16, bf16, bf16>(const HopArgs &, int, bool, int, cudaStream_t);
template cudaError_t launch_hop<bf16, float, bf16, bf16>(const HopArgs &, int, bool, int, cudaStream_t);

}  // namespace wd

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
#include "wd_internal.h"

namespace wd {

template <int MU, int SIGN, typename R>
__device__ __forceinline__ void spin_project(const cx<R> psi[12], cx<R> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<R> p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
        cx<R> a0, a1;   // A_mu (p2, p3)
        if (MU == 0)      { a0 = times_mi(p3); a1 = times_mi(p2); }          // A = -i s1
        else if (MU == 1) { a0 = cmake(-p3.re, -p3.im); a1 = p2; }           // A = -i s2
        else if (MU == 2) { a0 = times_mi(p2); a1 = times_i(p3); }           // A = -i s3
        else              { a0 = p2; a1 = p3; }                              // A = 1
        if (SIGN > 0) { h[c] = p0 + a0; h[3 + c] = p1 + a1; }
        else          { h[c] = p0 - a0; h[3 + c] = p1 - a1; }
    }
}

template <int MU, int SIGN, typename R>
__device__ __forceinline__ void spin_reconstruct_add(cx<R> acc[12], const cx<R> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<R> h0 = h[c], h1 = h[3 + c];
        acc[c] = acc[c] + h0;
        acc[3 + c] = acc[3 + c] + h1;
        cx<R> b0, b1;   // A_mu^dag (h0, h1)
        if (MU == 0)      { b0 = times_i(h1); b1 = times_i(h0); }
        else if (MU == 1) { b0 = h1; b1 = cmake(-h0.re, -h0.im); }
        else if (MU == 2) { b0 = times_i(h0); b1 = times_mi(h1); }
        else              { b0 = h0; b1 = h1; }
        if (SIGN > 0) { acc[6 + c] = acc[6 + c] + b0; acc[9 + c] = acc[9 + c] + b1; }
        else          { acc[6 + c] = acc[6 + c] - b0; acc[9 + c] = acc[9 + c] - b1; }
    }
}

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
        const int rhs = rb * R + r;
        if (rhs < A.nrhs) {
            cx<RT> psi[12], h[6], uh[6];
            SIO<SIn>::load((const uint4 *)A.in + (size_t)rhs * NCH * Vh, Vh, nb, psi);
            spin_project<MU, SIGN>(psi, h);
            su3_mul(u, h, uh);
            spin_reconstruct_add<MU, SIGN>(acc[r], uh);
        }
    }
}

template <typename SIn, typename SOut, typename SW, typename G, int R, bool DAG>
__global__ void __launch_bounds__(128) hop_kernel(HopArgs A) {
    typedef typename RealOf<SIn>::type RT;
    const int rb = blockIdx.x % A.nrb;
    const int s = (blockIdx.x / A.nrb) * blockDim.x + threadIdx.x;
    if (s >= A.g.Vh) return;
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
        const int rhs = rb * R + r;
        if (rhs >= A.nrhs) break;
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

template <typename SIn, typename SOut, typename SW, typename G>
cudaError_t launch_hop(const HopArgs &A0, int R, bool dag, int threads, cudaStream_t st) {
    HopArgs A = A0;
    if (A.nrhs <= 0) return cudaSuccess;
    if (R != 1 && R != 2 && R != 4) R = 1;
    A.nrb = (A.nrhs + R - 1) / R;
    const int sblocks = (A.g.Vh + threads - 1) / threads;
    dim3 grid((unsigned)(sblocks * A.nrb));
#define WD_HOP_CASE(RR)                                                                        \
    if (R == RR) {                                                                             \
        if (dag) hop_kernel<SIn, SOut, SW, G, RR, true><<<grid, threads, 0, st>>>(A);          \
        else hop_kernel<SIn, SOut, SW, G, RR, false><<<grid, threads, 0, st>>>(A);             \
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

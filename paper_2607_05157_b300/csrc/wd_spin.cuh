// Spin projection and reconstruction of the Wilson hop in the chiral basis,
// shared by every stencil variant (any real type with +, - and unary -).
//
// (1 -/+ g_mu) psi has rank 2: with g_mu = [[0, A_mu], [A_mu^dag, 0]] the hop
// needs only h = psi_up + sign*A_mu psi_down (6 complex), and the lower half of
// the result is sign*A_mu^dag (U h).  A_mu = -i s_k (k = 1, 2, 3), A_4 = 1.
#pragma once
#include "wd_common.cuh"

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

}  // namespace wd
